// amr.cu -- multi-block grids: static refinement (Sec. 3.2) and local
// adaptive time stepping (Sec. 3.4), batched over blocks.
//
// Device side: ghost zones are filled by sampling the neighbouring block
// that holds each ghost position (after mapping it across the receiving
// block's physical boundaries): a copy when the cell sizes agree, the
// average of the covered cells when the source is finer, the source cell
// plus offset x MINMOD slope when it is coarser (slopes whose stencil leaves
// the source interior are 0). A coarser-level source is interpolated in time
// between its old and new state; a same-level source is read at the same
// stage; a finer-level source, which has not yet advanced (coarse first), at
// its current state at both stages (the coarse fluxes through the shared
// faces are replaced by the finer ones at the end of the coarse step; an
// extrapolation in time to the coarse midpoint amplified step-to-step
// oscillations at coarse-fine faces of a magnetised torus).
//
// Same-level blocks stepped together share face fluxes (the coarser side
// takes the finer side's average) and edge EMFs (the dominant block's:
// finest cell along the edge, then finest across it, then lowest index).
// Across levels, a coarse step's boundary fluxes and EMFs are replaced at
// its end by the time integrals of the finer level's (refluxing), and its
// cells next to corrected faces are inverted again.
//
// Host side: the links (synchronisation entries, reflux records, refluxed
// cells) are built once; the launches of one period (2^Lmax fine substeps,
// levels coarsest first, every kernel batched over the due blocks of a
// level) are captured into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "grmhd.cuh"
#include "hamr_internal.h"

namespace hamr {
namespace {

constexpr int BSA = 128;
constexpr double PI_ = 3.14159265358979323846;

inline unsigned nb_(long n) { return (unsigned)((n + BSA - 1) / BSA); }

__host__ __device__ inline long pidx(const BlockView& v, int i, int j, int k) {
    return ((long)(k + NG) * v.n2p + (j + NG)) * v.n1p + (i + NG);
}

// ------------------------------------------------------------------ lookup
__host__ __device__ inline int find_block(const AmrDomain& A, const DevBlock* tab, const double x[4]) {
    int ib[4];
    for (int d = 1; d <= 3; d++) {
        double t = (x[d] - A.dlo[d]) / A.bkh[d] + 1e-6;  // a point on a plane belongs to the block above it
        int q = (int)floor(t);
        if (q < 0) {
            if (t < -1e-3) return -1;
            q = 0;
        }
        if (q >= A.nbk[d]) {
            if (t > A.nbk[d] + 1e-3) return -1;
            q = A.nbk[d] - 1;
        }
        ib[d] = q;
    }
    (void)tab;
    return A.bucket[((long)ib[3] * A.nbk[2] + ib[2]) * A.nbk[1] + ib[1]];
}

// maps x (outside block B) across B's physical boundaries; fdir = normal of a face point (0: cell centre)
__host__ __device__ inline void map_point(const AmrDomain& A, const DevBlock& B, double x[4], int fdir, int* neg,
                                          int* clamp) {
    *neg = 0;
    *clamp = 0;
    for (int d = 1; d <= 3; d++) {
        const double q = 0.25 * B.h[d];
        int side = -1;
        if (x[d] < B.lo[d] - q) side = 0;
        if (x[d] > B.hi[d] + q) side = 1;
        if (side < 0) continue;
        const int bc = B.v.bc[2 * (d - 1) + side];
        if (bc == HAMR_BC_OUTFLOW || bc == HAMR_BC_OUTFLOW_NOINFLOW) {
            if (d == fdir)
                x[d] = side ? B.hi[d] : B.lo[d];
            else
                x[d] = side ? B.hi[d] - 0.5 * B.h[d] : B.lo[d] + 0.5 * B.h[d];
            if (bc == HAMR_BC_OUTFLOW_NOINFLOW && d == 1) *clamp = side ? 1 : -1;
        } else if (bc == HAMR_BC_PERIODIC) {
            x[d] += side ? -(A.dhi[d] - A.dlo[d]) : (A.dhi[d] - A.dlo[d]);
        } else if (bc == HAMR_BC_POLAR) {
            x[2] = side ? 2.0 * PI_ - x[2] : -x[2];
            x[3] += PI_;
            *neg = 1;
        }
    }
    if (A.per[3]) {
        const double L = A.dhi[3] - A.dlo[3];
        while (x[3] >= A.dhi[3] - 1e-12 * L) x[3] -= L;
        while (x[3] < A.dlo[3] - 1e-12 * L) x[3] += L;
    }
}

// per-dimension footprint of a target cell (size ht, centre x) in block N
__host__ __device__ inline void footprint(const DevBlock& N, const double x[4], const double ht[4], int i0[4],
                                          int cnt[4], double dl[4]) {
    for (int d = 1; d <= 3; d++) {
        const double hs = N.h[d];
        const double r = ht[d] / hs;
        dl[d] = 0.0;
        if (r > 1.5) {
            cnt[d] = (int)llround(r);
            i0[d] = (int)llround((x[d] - 0.5 * ht[d] - N.lo[d]) / hs);
        } else {
            cnt[d] = 1;
            i0[d] = (int)floor((x[d] - N.lo[d]) / hs);
            if (r < 0.75) dl[d] = nearbyint(8.0 * (x[d] - (N.lo[d] + (i0[d] + 0.5) * hs)) / hs) / 8.0;
        }
    }
}

// the source state seen by receiver R at stage sigma of substep s
struct SrcView {
    const double *Pa, *Pb, *Ba, *Bb;
    double w;
    __device__ double P(long i) const { return Pb ? Pa[i] + w * (Pb[i] - Pa[i]) : Pa[i]; }
    __device__ double B(long i) const { return Bb ? Ba[i] + w * (Bb[i] - Ba[i]) : Ba[i]; }
};

// 2^e as a double, built from its bits (-1022 <= e <= 1023): exact, and no work for the FP64 pipe
__device__ inline double pow2i(int e) { return __hiloint2double((1023 + e) << 20, 0); }

__device__ inline SrcView source_view(const DevBlock& R, const DevBlock& N, int sigma, int s) {
    SrcView v;
    v.Pb = v.Bb = nullptr;
    v.w = 0.0;
    if (N.lat > R.lat) {
        // w = (s - s0 + sigma 2^Lr / 2) / 2^Ln = (2 (s - s0) + sigma 2^Lr) 2^-(Ln+1), exact
        const int s0 = (s >> N.lat) << N.lat;
        const int k = 2 * (s - s0) + sigma * (1 << R.lat);
        v.Pa = N.Pold;
        v.Ba = N.Bold;
        if (k != 0) {  // else the source's old state itself
            v.Pb = N.P;
            v.Bb = N.B;
            v.w = (double)k * pow2i(-(N.lat + 1));
        }
    } else if (N.lat == R.lat && sigma == 1) {
        v.Pa = N.Ph;
        v.Ba = N.Bh;
    } else {  // same level at the predictor, or finer: its current state
        v.Pa = N.P;
        v.Ba = N.B;
    }
    return v;
}

// MINMOD: the argument of smaller magnitude where both have the same strict sign, else 0. On the
// bit patterns (the order of non-negative doubles is that of their patterns as integers), so
// that it costs the FP64 pipe nothing
__device__ inline double minmod_(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
    if ((ia ^ ib) < 0 || ma == 0 || mb == 0) return 0.0;
    return ma < mb ? a : b;
}

// 1 / (c1 c2 c3) for footprint counts: built from its bits when the product is a power of two
// (every footprint of a 2:1 tree), else divided
__device__ inline double inv_count(int c1, int c2, int c3) {
    const int p = c1 * c2 * c3;
    if ((p & (p - 1)) == 0) return pow2i(-(31 - __clz(p)));
    return 1.0 / (double)p;
}

// ------------------------------------------------------------------ ghost kernels
// A ghost cell or face first locates its source (the block holding the mapped
// point, the footprint there, the prolongation offsets and the sign flips of
// the polar map), then forms its value from the source's state at the stage's
// time. The location depends only on the tree, so the grid stores it once per
// ghost (GhostLoc, built by k_ghost_*_locate with the same device code) and
// the stage launches only apply it; the direct kernels (locate and apply in
// one) remain for trees whose footprints do not fit the packed form.

// packed location of one ghost: receiving padded index t, source block n (-1: none),
// base padded index c0 of the footprint in n, and in pk: footprint counts (4 bits each,
// bits 0..11), offsets in eighths of a source cell (signed 4 bits each, bits 12..23:
// the prolongation offsets dl of a cell, the face fraction fr in the face's normal
// slot), the polar sign flip (bit 24), the radial no-inflow clamp of u^1 (bits 25..26:
// 1 keeps it >= 0, 2 keeps it <= 0) and the face direction (bits 28..29)
struct GhostLoc {
    int t, n, c0;
    unsigned pk;
};

struct GhostGeo {  // an unpacked location
    int n, cnt[4], e8[4], neg, clamp, fd;
    long c0;
};

__device__ inline bool pack_loc(const GhostGeo& G, int t, GhostLoc& L) {
    L.t = t;
    L.n = G.n;
    L.c0 = (int)G.c0;
    unsigned pk = 0;
    bool ok = G.c0 >= 0 && G.c0 < 0x7FFFFFFF;
    for (int d = 1; d <= 3; d++) {
        ok = ok && G.cnt[d] >= 1 && G.cnt[d] <= 15 && G.e8[d] >= -7 && G.e8[d] <= 7;
        pk |= (unsigned)(G.cnt[d] & 15) << (4 * (d - 1));
        pk |= (unsigned)(G.e8[d] & 15) << (12 + 4 * (d - 1));
    }
    pk |= (unsigned)(G.neg & 1) << 24;
    pk |= (unsigned)(G.clamp > 0 ? 1 : (G.clamp < 0 ? 2 : 0)) << 25;
    pk |= (unsigned)(G.fd & 3) << 28;
    L.pk = pk;
    return ok || G.n < 0;
}

__device__ inline void unpack_loc(const GhostLoc& L, GhostGeo& G) {
    G.n = L.n;
    G.c0 = L.c0;
    for (int d = 1; d <= 3; d++) {
        G.cnt[d] = (int)((L.pk >> (4 * (d - 1))) & 15u);
        const int e = (int)((L.pk >> (12 + 4 * (d - 1))) & 15u);
        G.e8[d] = (e & 8) ? e - 16 : e;
    }
    G.neg = (int)((L.pk >> 24) & 1u);
    const unsigned c = (L.pk >> 25) & 3u;
    G.clamp = (c == 1u) ? 1 : ((c == 2u) ? -1 : 0);
    G.fd = (int)((L.pk >> 28) & 3u);
}

// the source of ghost cell (i, j, k) of R; G.n = -1 where no block holds the mapped point.
// e8[d]: the MINMOD prolongation offset in eighths, 0 where the slope stencil leaves the
// source block's interior (the value then takes no slope in d)
__device__ inline void ghost_cell_locate(const AmrDomain& A, const DevBlock& R, int i, int j, int k, GhostGeo& G) {
    double x[4] = {0.0, R.lo[1] + (i + 0.5) * R.h[1], R.lo[2] + (j + 0.5) * R.h[2], R.lo[3] + (k + 0.5) * R.h[3]};
    int neg, clamp;
    map_point(A, R, x, 0, &neg, &clamp);
    G.n = find_block(A, A.tab, x);
    G.neg = neg;
    G.clamp = clamp;
    G.fd = 0;
    if (G.n < 0) {
        G.c0 = 0;
        for (int d = 1; d <= 3; d++) G.cnt[d] = 1, G.e8[d] = 0;
        return;
    }
    const DevBlock& N = A.tab[G.n];
    int i0[4];
    double dl[4];
    footprint(N, x, R.h, i0, G.cnt, dl);
    const int nn[4] = {0, N.v.n1, N.v.n2, N.v.n3};
    for (int d = 1; d <= 3; d++) {
        G.e8[d] = (int)(8.0 * dl[d]);  // dl is a multiple of 1/8
        if (i0[d] - 1 < 0 || i0[d] + 1 >= nn[d]) G.e8[d] = 0;
    }
    G.c0 = pidx(N.v, i0[1], i0[2], i0[3]);
}

// the value of a located ghost cell at stage sigma of substep s into P (or Ph) of R at t
__device__ inline void ghost_cell_apply(const AmrDomain& A, const DevBlock& R, const GhostGeo& G, long t, int sigma,
                                        int s) {
    if (G.n < 0) return;
    const DevBlock& N = A.tab[G.n];
    const SrcView S = source_view(R, N, sigma, s);
    const long sj = N.v.n1p, sk = (long)N.v.n1p * N.v.n2p;
    const long st[4] = {0, 1, sj, sk};
    const bool one = G.cnt[1] * G.cnt[2] * G.cnt[3] == 1;
    const double inv = inv_count(G.cnt[1], G.cnt[2], G.cnt[3]);
    double f[4];  // the prolongation offsets in source cells (multiples of 1/8: exact)
    for (int d = 1; d <= 3; d++) f[d] = (G.e8[d] == 0) ? 0.0 : (double)G.e8[d] * 0.125;
    double* out = sigma ? R.Ph : R.P;
    // source cell c of primitive q, with its MINMOD slopes where prolonged
    auto cell = [&](int q, long c) {
        const double q0 = S.P(q * N.v.nc + c);
        double val = q0;
        for (int d = 1; d <= 3; d++) {
            if (G.e8[d] == 0) continue;
            const double qm = S.P(q * N.v.nc + c - st[d]);
            const double qp = S.P(q * N.v.nc + c + st[d]);
            val += f[d] * minmod_(q0 - qm, qp - q0);
        }
        return val;
    };
    // every primitive is formed before any is stored, so that the gathers of all eight are in
    // flight together (a store between them could alias the next source and would serialise them)
    double ov[NPRIM];
    if (one) {  // a copy or a prolongation: one source cell, no sum
#pragma unroll
        for (int q = 0; q < NPRIM; q++) ov[q] = cell(q, G.c0);
    } else {  // the mean of the covered finer cells
#pragma unroll
        for (int q = 0; q < NPRIM; q++) {
            double sum = 0.0;
            for (int c3 = 0; c3 < G.cnt[3]; c3++)
                for (int c2 = 0; c2 < G.cnt[2]; c2++)
                    for (int c1 = 0; c1 < G.cnt[1]; c1++) sum += cell(q, G.c0 + c1 + c2 * sj + c3 * sk);
            ov[q] = sum * inv;
        }
    }
#pragma unroll
    for (int q = 0; q < NPRIM; q++) {
        double o = ov[q];
        if (G.neg && (q == U2 || q == B2)) o = -o;
        if (q == U1) {
            if (G.clamp > 0 && o < 0.0) o = 0.0;
            if (G.clamp < 0 && o > 0.0) o = 0.0;
        }
        out[q * R.v.nc + t] = o;
    }
}

// the source of ghost face (i, j, k) of direction fd of R: the face fraction fr (eighths of a
// source face spacing toward the next face) in e8[fd]
__device__ inline void ghost_face_locate(const AmrDomain& A, const DevBlock& R, int fd, int i, int j, int k,
                                         GhostGeo& G) {
    const int ii[4] = {0, i, j, k};
    double x[4] = {0.0, R.lo[1] + (i + 0.5) * R.h[1], R.lo[2] + (j + 0.5) * R.h[2], R.lo[3] + (k + 0.5) * R.h[3]};
    x[fd] = R.lo[fd] + ii[fd] * R.h[fd];
    int neg, clamp;
    map_point(A, R, x, fd, &neg, &clamp);
    G.n = find_block(A, A.tab, x);
    G.neg = neg;
    G.clamp = 0;
    G.fd = fd;
    if (G.n < 0) {
        G.c0 = 0;
        for (int d = 1; d <= 3; d++) G.cnt[d] = 1, G.e8[d] = 0;
        return;
    }
    const DevBlock& N = A.tab[G.n];
    int i0[4];
    double dl[4];
    double xc[4] = {0.0, x[1], x[2], x[3]};
    xc[fd] += 0.5 * R.h[fd];
    footprint(N, xc, R.h, i0, G.cnt, dl);
    const double pos = (x[fd] - N.lo[fd]) / N.h[fd];
    int p0 = (int)floor(pos + 1e-9);
    double fr = nearbyint(8.0 * (pos - p0)) / 8.0;
    if (fr >= 1.0) {
        p0 += 1;
        fr = 0.0;
    }
    G.cnt[fd] = 1;
    i0[fd] = p0;
    for (int d = 1; d <= 3; d++) G.e8[d] = 0;
    G.e8[fd] = (int)(8.0 * fr);
    G.c0 = pidx(N.v, i0[1], i0[2], i0[3]);
}

__device__ inline void ghost_face_apply(const AmrDomain& A, const DevBlock& R, const GhostGeo& G, long t, int sigma,
                                        int s) {
    if (G.n < 0) return;
    const DevBlock& N = A.tab[G.n];
    const SrcView S = source_view(R, N, sigma, s);
    const int fd = G.fd;
    const long sj = N.v.n1p, sk = (long)N.v.n1p * N.v.n2p;
    const long st = (fd == 1) ? 1 : ((fd == 2) ? sj : sk);
    const int e8 = G.e8[fd];
    const double fr = (e8 == 0) ? 0.0 : (double)e8 * 0.125;
    const bool one = G.cnt[1] * G.cnt[2] * G.cnt[3] == 1;
    const double inv = inv_count(G.cnt[1], G.cnt[2], G.cnt[3]);
    auto face = [&](long c) {  // source face c, linear toward the next where between two
        double q = S.B((fd - 1) * N.v.nc + c);
        if (e8 != 0) {
            const double q1 = S.B((fd - 1) * N.v.nc + c + st);
            q = q + fr * (q1 - q);
        }
        return q;
    };
    double val;
    if (one) {
        val = face(G.c0);
    } else {
        double sum = 0.0;
        for (int c3 = 0; c3 < G.cnt[3]; c3++)
            for (int c2 = 0; c2 < G.cnt[2]; c2++)
                for (int c1 = 0; c1 < G.cnt[1]; c1++) sum += face(G.c0 + c1 + c2 * sj + c3 * sk);
        val = sum * inv;
    }
    double* out = sigma ? R.Bh : R.B;
    out[(fd - 1) * R.v.nc + t] = (G.neg && fd == 2) ? -val : val;
}

// padded cell t of R as (i, j, k); false for an interior cell
__device__ inline bool ghost_cell_at(const BlockView& v, long t, int& i, int& j, int& k) {
    i = (int)(t % v.n1p) - NG;
    j = (int)((t / v.n1p) % v.n2p) - NG;
    k = (int)(t / ((long)v.n1p * v.n2p)) - NG;
    return !(i >= 0 && i < v.n1 && j >= 0 && j < v.n2 && k >= 0 && k < v.n3);
}

// padded face t of direction fd of R as (i, j, k); false for a face the block owns
__device__ inline bool ghost_face_at(const BlockView& v, int fd, long t, int& i, int& j, int& k) {
    i = (int)(t % v.n1p) - NG;
    j = (int)((t / v.n1p) % v.n2p) - NG;
    k = (int)(t / ((long)v.n1p * v.n2p)) - NG;
    const int ii[4] = {0, i, j, k};
    const int nn[4] = {0, v.n1, v.n2, v.n3};
    for (int e = 1; e <= 3; e++) {
        if (e == fd) {
            if (ii[e] < 0 || ii[e] > nn[e]) return true;
        } else if (ii[e] < 0 || ii[e] >= nn[e]) {
            return true;
        }
    }
    return false;
}

// direct forms: locate and apply per launch
__global__ void k_ghost_cells(AmrDomain A, const int* list, int sigma, int s) {
    const DevBlock& R = A.tab[list[blockIdx.y]];
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)R.v.n1p * R.v.n2p * R.v.n3p) return;
    int i, j, k;
    if (!ghost_cell_at(R.v, t, i, j, k)) return;
    GhostGeo G;
    ghost_cell_locate(A, R, i, j, k, G);
    ghost_cell_apply(A, R, G, t, sigma, s);
}

__global__ void k_ghost_faces(AmrDomain A, const int* list, int sigma, int s) {
    const DevBlock& R = A.tab[list[blockIdx.y]];
    const long np = (long)R.v.n1p * R.v.n2p * R.v.n3p;
    const long tt = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tt >= 3 * np) return;
    const int fd = 1 + (int)(tt / np);
    const long t = tt % np;
    int i, j, k;
    if (!ghost_face_at(R.v, fd, t, i, j, k)) return;
    GhostGeo G;
    ghost_face_locate(A, R, fd, i, j, k, G);
    ghost_face_apply(A, R, G, t, sigma, s);
}

// stored locations: the builders take entry (t, receiving block) and fill the rest;
// *bad counts entries whose footprint does not fit the packed form
__global__ void k_ghost_cells_locate(AmrDomain A, GhostLoc* loc, long n, int* bad) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const DevBlock& R = A.tab[loc[q].n];
    const long t = loc[q].t;
    int i, j, k;
    ghost_cell_at(R.v, t, i, j, k);
    GhostGeo G;
    ghost_cell_locate(A, R, i, j, k, G);
    if (!pack_loc(G, (int)t, loc[q])) atomicAdd(bad, 1);
}

__global__ void k_ghost_faces_locate(AmrDomain A, GhostLoc* loc, long n, int* bad) {
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const DevBlock& R = A.tab[loc[q].n];
    const int fd = (int)(loc[q].pk >> 28) & 3;
    const long t = loc[q].t;
    int i, j, k;
    ghost_face_at(R.v, fd, t, i, j, k);
    GhostGeo G;
    ghost_face_locate(A, R, fd, i, j, k, G);
    if (!pack_loc(G, (int)t, loc[q])) atomicAdd(bad, 1);
}

// the stage launches: ghost g of block list[blockIdx.y] (gofs / gcnt: the block's entries)
__global__ void k_ghost_cells_mapped(AmrDomain A, const int* list, int sigma, int s, const GhostLoc* loc) {
    const DevBlock& R = A.tab[list[blockIdx.y]];
    const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= R.ng_cell) return;
    const GhostLoc L = loc[R.gofs_cell + g];
    GhostGeo G;
    unpack_loc(L, G);
    ghost_cell_apply(A, R, G, L.t, sigma, s);
}

__global__ void k_ghost_faces_mapped(AmrDomain A, const int* list, int sigma, int s, const GhostLoc* loc) {
    const DevBlock& R = A.tab[list[blockIdx.y]];
    const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= R.ng_face) return;
    const GhostLoc L = loc[R.gofs_face + g];
    GhostGeo G;
    unpack_loc(L, G);
    ghost_face_apply(A, R, G, L.t, sigma, s);
}

// ------------------------------------------------------------------ regridding
// The state of a new tree from the old one (Sec. 3.2: prolongation and
// restriction on (de)refinement). Cell-centred primitives are sampled like
// ghosts from the old block holding the cell centre (copy, volume average or
// MINMOD-limited prolongation; primitives, the paper's faster and more
// robust choice). Face fields: copy, area average, or from an old coarser
// block the divergence-free reconstruction of Balsara (2001): a field
// quadratic in the coarse cell's local coordinates that is exactly
// divergence-free and matches each coarse face's mean and MINMOD-limited
// tangential slopes (0 where the stencil leaves the old block's faces); a
// fine face takes it at its centre. Where a coarse cell borders old finer
// data, the fine faces on that coarse face are the old fine faces and the
// cell's interior fine faces are corrected (least change) so that each fine
// cell stays divergence-free. A face on a plane between two old blocks is
// taken from the finer one.

__device__ inline void wrap_domain(const AmrDomain& A, double x[4]) {
    for (int d = 1; d <= 3; d++) {
        if (!A.per[d]) continue;
        const double L = A.dhi[d] - A.dlo[d];
        while (x[d] >= A.dhi[d]) x[d] -= L;
        while (x[d] < A.dlo[d]) x[d] += L;
    }
}

__global__ void k_regrid_cells(AmrDomain A, const DevBlock* ntab) {
    const DevBlock& R = ntab[blockIdx.y];
    const BlockView& v = R.v;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)v.n1 * v.n2 * v.n3) return;
    const int i = (int)(t % v.n1), j = (int)((t / v.n1) % v.n2), k = (int)(t / ((long)v.n1 * v.n2));
    double x[4] = {0.0, R.lo[1] + (i + 0.5) * R.h[1], R.lo[2] + (j + 0.5) * R.h[2], R.lo[3] + (k + 0.5) * R.h[3]};
    const int n = find_block(A, A.tab, x);
    if (n < 0) return;
    const DevBlock& N = A.tab[n];
    int i0[4], cnt[4];
    double dl[4];
    footprint(N, x, R.h, i0, cnt, dl);
    const int nn[4] = {0, N.v.n1, N.v.n2, N.v.n3};
    const double inv = 1.0 / (double)(cnt[1] * cnt[2] * cnt[3]);
    const long c = pidx(v, i, j, k);
    for (int q = 0; q < 5; q++) {
        double sum = 0.0;
        for (int c3 = 0; c3 < cnt[3]; c3++)
            for (int c2 = 0; c2 < cnt[2]; c2++)
                for (int c1 = 0; c1 < cnt[1]; c1++) {
                    const int ii[4] = {0, i0[1] + c1, i0[2] + c2, i0[3] + c3};
                    const long cs = pidx(N.v, ii[1], ii[2], ii[3]);
                    const double q0 = N.P[q * N.v.nc + cs];
                    double val = q0;
                    for (int d = 1; d <= 3; d++) {
                        if (dl[d] == 0.0) continue;
                        if (ii[d] - 1 < 0 || ii[d] + 1 >= nn[d]) continue;
                        const long st = (d == 1) ? 1 : ((d == 2) ? (long)N.v.n1p : (long)N.v.n1p * N.v.n2p);
                        val += dl[d] * minmod_(q0 - N.P[q * N.v.nc + cs - st], N.P[q * N.v.nc + cs + st] - q0);
                    }
                    sum += val;
                }
        R.P[q * v.nc + c] = sum * inv;
    }
}

// tangential MINMOD slope of face field a of block N at face ii along b, per unit local coordinate
__device__ inline double face_slope(const DevBlock& N, int a, const int ii[4], int b) {
    const int nn[4] = {0, N.v.n1, N.v.n2, N.v.n3};
    if (ii[b] - 1 < 0 || ii[b] + 1 > nn[b] - 1) return 0.0;
    const long st = (b == 1) ? 1 : ((b == 2) ? (long)N.v.n1p : (long)N.v.n1p * N.v.n2p);
    const double* B = N.B + (long)(a - 1) * N.v.nc;
    const long c = pidx(N.v, ii[1], ii[2], ii[3]);
    const double q0 = B[c];
    return 0.5 * minmod_(q0 - B[c - st], B[c + st] - q0);
}

// the coarse cell of N holding `probe` and the local coordinates (-1..1) of x in it
__device__ inline void coarse_cell(const DevBlock& N, const double x[4], const double probe[4], int ic[4],
                                   double xi[4]) {
    const int nn[4] = {0, N.v.n1, N.v.n2, N.v.n3};
    for (int d = 1; d <= 3; d++) {
        ic[d] = (int)floor((probe[d] - N.lo[d]) / N.h[d]);
        ic[d] = min(max(ic[d], 0), nn[d] - 1);
        xi[d] = 2.0 * (x[d] - (N.lo[d] + (ic[d] + 0.5) * N.h[d])) / N.h[d];
    }
}

// Balsara's divergence-free polynomial of face component fd in coarse cell ic of N at local coordinates xi
__device__ inline double balsara_poly(const DevBlock& N, const int ic[4], const double xi[4], int fd) {
    double Fm[4], Fp[4], Sm[4][4], Sp[4][4];
    for (int a = 1; a <= 3; a++) {
        int lo[4] = {0, ic[1], ic[2], ic[3]}, hi[4] = {0, ic[1], ic[2], ic[3]};
        hi[a]++;
        const double* B = N.B + (long)(a - 1) * N.v.nc;
        Fm[a] = B[pidx(N.v, lo[1], lo[2], lo[3])];
        Fp[a] = B[pidx(N.v, hi[1], hi[2], hi[3])];
        for (int b = 1; b <= 3; b++) {
            Sm[a][b] = Sp[a][b] = 0.0;
            if (b == a) continue;
            Sm[a][b] = face_slope(N, a, lo, b);
            Sp[a][b] = face_slope(N, a, hi, b);
        }
    }
    const int a = fd;
    double Aaa = 0.0;
    for (int b = 1; b <= 3; b++)
        if (b != a) Aaa += 0.5 * (Sp[b][a] - Sm[b][a]) / N.h[b];
    Aaa *= -0.5 * N.h[a];
    double val = 0.5 * (Fp[a] + Fm[a]) - Aaa + 0.5 * (Fp[a] - Fm[a]) * xi[a] + Aaa * xi[a] * xi[a];
    for (int b = 1; b <= 3; b++) {
        if (b == a) continue;
        val += 0.5 * (Sp[a][b] + Sm[a][b]) * xi[b] + 0.5 * (Sp[a][b] - Sm[a][b]) * xi[a] * xi[b];
    }
    return val;
}

__device__ inline double sample_face_plain(const DevBlock& N, const double x[4], const double ht[4], int fd);

// cell widths a narrower than b in some direction (a block finer than b along it)
__device__ inline bool finer_cells(const double a[4], const double b[4]) {
    return a[1] < b[1] * (1.0 - 1e-9) || a[2] < b[2] * (1.0 - 1e-9) || a[3] < b[3] * (1.0 - 1e-9);
}
__device__ inline double cell_volume(const double h[4]) { return h[1] * h[2] * h[3]; }

// refinement factor (1 or 2) per direction of new cells of widths hn inside the old coarser block N: an
// octree child halves all three widths, a 6-way polar child on the axis keeps N's x3 width
__device__ inline void refine_factors(const DevBlock& N, const double hn[4], int f[4]) {
    f[0] = 1;
    for (int d = 1; d <= 3; d++) f[d] = (N.h[d] > 1.5 * hn[d]) ? 2 : 1;
}

// a fine face (cell widths hn) on coarse face (a, side) of cell ic; along each tangential direction b < c
// one of its two halves (tb, tc) where the refinement splits that direction, else the whole width
// (tb, tc = 0): the old tree's finer data beyond it, else the face's linear profile
__device__ inline double fine_face_on_coarse(const AmrDomain& A, const DevBlock& N, const int ic[4], int a,
                                             int side, int tb, int tc, const double hn[4]) {
    const int b = (a == 1) ? 2 : 1, c = (a == 3) ? 2 : 3;
    int f[4];
    refine_factors(N, hn, f);
    const double ob = (f[b] == 2) ? 0.25 + 0.5 * tb : 0.5, oc = (f[c] == 2) ? 0.25 + 0.5 * tc : 0.5;
    double x[4];
    x[0] = 0.0;
    x[a] = N.lo[a] + (ic[a] + side) * N.h[a];
    x[b] = N.lo[b] + (ic[b] + ob) * N.h[b];
    x[c] = N.lo[c] + (ic[c] + oc) * N.h[c];
    double probe[4] = {0.0, x[1], x[2], x[3]};
    probe[a] += (side ? 0.25 : -0.25) * hn[a];
    wrap_domain(A, probe);
    const int n = find_block(A, A.tab, probe);
    if (n >= 0 && finer_cells(A.tab[n].h, N.h)) {
        double xs[4] = {0.0, probe[1], probe[2], probe[3]};
        xs[a] -= (side ? 0.25 : -0.25) * hn[a];
        const DevBlock& B = A.tab[n];
        if (B.h[b] > 1.5 * hn[b] || B.h[c] > 1.5 * hn[c]) {
            // its cells wider than the new face along the plane: its polynomial's linear profile on its
            // face, the value the new block on the other side of the plane takes for this face
            int icb[4];
            double xib[4];
            coarse_cell(B, xs, probe, icb, xib);
            return balsara_poly(B, icb, xib, a);
        }
        return sample_face_plain(B, xs, hn, a);
    }
    double xi[4] = {0.0, 0.0, 0.0, 0.0};
    xi[a] = side ? 1.0 : -1.0;
    xi[b] = (f[b] == 2) ? (tb ? 0.5 : -0.5) : 0.0;
    xi[c] = (f[c] == 2) ? (tc ? 0.5 : -0.5) : 0.0;
    return balsara_poly(N, ic, xi, a);
}

// a fine face interior to coarse cell ic (local plane xi_fd = 0), the cell split into f1 x f2 x f3 fine
// cells (2 x 2 x 2 for an octree child, 2 x 2 x 1 for a polar child on the axis): the polynomial's value
// corrected by the least change of the interior faces that makes every fine cell divergence-free, given
// the fine faces on the cell's boundary. The fine cells' graph Laplacian L (weights A_d^2 along the split
// directions, A_d the fine face areas) has the parity vectors chi_s(c) = (-1)^(s.c), s a subset of the
// split directions, as eigenvectors with eigenvalues 2 sum_d s_d A_d^2, so L lambda = -D is solved in
// closed form; the change across an interior face of direction d is A_d (lambda_lo - lambda_hi).
__device__ inline double interior_fine_face(const AmrDomain& A, const DevBlock& N, const int ic[4],
                                            const double xi[4], int fd, const double hn[4]) {
    int f[4];
    refine_factors(N, hn, f);
    double F[4][3][2][2];
    for (int a = 1; a <= 3; a++) {
        const int b = (a == 1) ? 2 : 1, c = (a == 3) ? 2 : 3;
        for (int tb = 0; tb < f[b]; tb++)
            for (int tc = 0; tc < f[c]; tc++) {
                F[a][0][tb][tc] = fine_face_on_coarse(A, N, ic, a, 0, tb, tc, hn);
                F[a][2][tb][tc] = fine_face_on_coarse(A, N, ic, a, 1, tb, tc, hn);
                if (f[a] == 2) {
                    double x0[4] = {0.0, 0.0, 0.0, 0.0};
                    x0[b] = (f[b] == 2) ? (tb ? 0.5 : -0.5) : 0.0;
                    x0[c] = (f[c] == 2) ? (tc ? 0.5 : -0.5) : 0.0;
                    F[a][1][tb][tc] = balsara_poly(N, ic, x0, a);
                }
            }
    }
    const double Ar[4] = {0.0, hn[2] * hn[3], hn[1] * hn[3], hn[1] * hn[2]};
    // split directions as a bit mask; the fine cells are the c with no bit outside it
    const int smask = (f[1] == 2 ? 1 : 0) | (f[2] == 2 ? 2 : 0) | (f[3] == 2 ? 4 : 0);
    const double ncell = (double)(f[1] * f[2] * f[3]);
    double D[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < 8; c++) {
        if (c & ~smask) continue;
        const int ix[4] = {0, c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double sum = 0.0;
        for (int a = 1; a <= 3; a++) {
            const int b = (a == 1) ? 2 : 1, cc = (a == 3) ? 2 : 3;
            const int lo = (f[a] == 2) ? ix[a] : 0, up = (f[a] == 2) ? ix[a] + 1 : 2;
            sum += Ar[a] * (F[a][up][ix[b]][ix[cc]] - F[a][lo][ix[b]][ix[cc]]);
        }
        D[c] = sum;
    }
    // lambda = sum_{s != 0, s within the split directions} (rho_s / mu_s) chi_s, rho_s = (1/n) sum_c chi_s(c) (-D_c)
    double lam[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int sm = 1; sm < 8; sm++) {
        if (sm & ~smask) continue;
        double rho = 0.0;
        for (int c = 0; c < 8; c++)
            if (!(c & ~smask)) rho -= (__popc(sm & c) & 1) ? -D[c] : D[c];
        rho /= ncell;
        double mu = 0.0;
        for (int a = 1; a <= 3; a++)
            if (sm & (1 << (a - 1))) mu += 2.0 * Ar[a] * Ar[a];
        const double coef = rho / mu;
        for (int c = 0; c < 8; c++)
            if (!(c & ~smask)) lam[c] += (__popc(sm & c) & 1) ? -coef : coef;
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
    return F[fd][1][tb][tc] + Ar[fd] * (lam[clo] - lam[chi]);
}

// face field fd of a target face (cell size ht) at x from a source of the same or finer size
__device__ inline double sample_face_plain(const DevBlock& N, const double x[4], const double ht[4], int fd) {
    int i0[4], cnt[4];
    double dl[4];
    double xc[4] = {0.0, x[1], x[2], x[3]};
    xc[fd] += 0.5 * ht[fd];
    footprint(N, xc, ht, i0, cnt, dl);
    const double pos = (x[fd] - N.lo[fd]) / N.h[fd];
    int p0 = (int)floor(pos + 1e-9);
    double fr = nearbyint(8.0 * (pos - p0)) / 8.0;
    if (fr >= 1.0) {
        p0 += 1;
        fr = 0.0;
    }
    cnt[fd] = 1;
    const double inv = 1.0 / (double)(cnt[1] * cnt[2] * cnt[3]);
    const long st = (fd == 1) ? 1 : ((fd == 2) ? (long)N.v.n1p : (long)N.v.n1p * N.v.n2p);
    const double* B = N.B + (long)(fd - 1) * N.v.nc;
    double sum = 0.0;
    for (int c3 = 0; c3 < cnt[3]; c3++)
        for (int c2 = 0; c2 < cnt[2]; c2++)
            for (int c1 = 0; c1 < cnt[1]; c1++) {
                int jj[4] = {0, i0[1] + c1, i0[2] + c2, i0[3] + c3};
                jj[fd] = p0;
                const long c = pidx(N.v, jj[1], jj[2], jj[3]);
                double q = B[c];
                if (fr != 0.0) q = q + fr * (B[c + st] - q);
                sum += q;
            }
    return sum * inv;
}

__global__ void k_regrid_faces(AmrDomain A, const DevBlock* ntab) {
    const DevBlock& R = ntab[blockIdx.y];
    const BlockView& v = R.v;
    const long nf = (long)(v.n1 + 1) * (v.n2 + 1) * (v.n3 + 1);
    const long tt = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tt >= 3 * nf) return;
    const int fd = 1 + (int)(tt / nf);
    const long t = tt % nf;
    const int i = (int)(t % (v.n1 + 1)), j = (int)((t / (v.n1 + 1)) % (v.n2 + 1)),
              k = (int)(t / ((long)(v.n1 + 1) * (v.n2 + 1)));
    const int ii[4] = {0, i, j, k};
    const int nn[4] = {0, v.n1, v.n2, v.n3};
    for (int e = 1; e <= 3; e++)
        if (e != fd && ii[e] >= nn[e]) return;  // only the block's own faces
    double x[4] = {0.0, R.lo[1] + (i + 0.5) * R.h[1], R.lo[2] + (j + 0.5) * R.h[2], R.lo[3] + (k + 0.5) * R.h[3]};
    x[fd] = R.lo[fd] + ii[fd] * R.h[fd];
    double pl[4] = {0.0, x[1], x[2], x[3]}, pr[4] = {0.0, x[1], x[2], x[3]};
    pl[fd] -= 0.25 * R.h[fd];
    pr[fd] += 0.25 * R.h[fd];
    wrap_domain(A, pl);
    wrap_domain(A, pr);
    const int nl = find_block(A, A.tab, pl), nr = find_block(A, A.tab, pr);
    int n = nr;
    bool left = false;
    if (n < 0 || (nl >= 0 && cell_volume(A.tab[nl].h) < cell_volume(A.tab[nr].h) * (1.0 - 1e-9))) {
        n = nl;
        left = true;
    }
    if (n < 0) return;
    const DevBlock& N = A.tab[n];
    const double* probe = left ? pl : pr;
    double xs[4] = {0.0, probe[1], probe[2], probe[3]};
    xs[fd] += (left ? 0.25 : -0.25) * R.h[fd];
    double val;
    if (N.h[1] > R.h[1] * 1.5 || N.h[2] > R.h[2] * 1.5 || N.h[3] > R.h[3] * 1.5) {
        int ic[4];
        double xi[4];
        coarse_cell(N, xs, probe, ic, xi);
        val = (fabs(xi[fd]) > 0.5) ? balsara_poly(N, ic, xi, fd) : interior_fine_face(A, N, ic, xi, fd, R.h);
    } else {
        val = sample_face_plain(N, xs, R.h, fd);
    }
    R.B[(long)(fd - 1) * v.nc + pidx(v, i, j, k)] = val;
}

// ------------------------------------------------------------------ synchronisation
struct SyncDev {  // SoA: dst block, field/face direction, dst index, source block, n <= 4 source indices
    const int *dst, *dir, *src, *n;
    const long *di, *si;
};

// flux32: the destination's FP32 copies of the field slots 6 and 7 (kept after its FP64 fields for
// the FP32 EMFs) follow the synchronised values
__global__ void k_flux_sync(const DevBlock* tab, SyncDev S, int beg, int end, int flux32) {
    const int e = beg + (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= end) return;
    const DevBlock& D = tab[S.dst[e]];
    const DevBlock& F = tab[S.src[e]];
    const int d = S.dir[e];
    double* Fd = (d == 1) ? D.F1 : ((d == 2) ? D.F2 : D.F3);
    const double* Fs = (d == 1) ? F.F1 : ((d == 2) ? F.F2 : F.F3);
    const int n = S.n[e];
    const double inv = 1.0 / (double)n;
    for (int q = 0; q < NFLUX; q++) {
        double sum = 0.0;
        for (int m = 0; m < n; m++) sum += Fs[q * F.v.nc + S.si[4 * e + m]];
        Fd[q * D.v.nc + S.di[e]] = sum * inv;
        if (flux32 && q >= 6)
            reinterpret_cast<float*>(Fd + NFLUX * D.v.nc)[(q - 6) * D.v.nc + S.di[e]] = (float)(sum * inv);
    }
}

__global__ void k_edge_gather(const DevBlock* tab, SyncDev S, int beg, int end, double* tmp) {
    const int e = beg + (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= end) return;
    const DevBlock& F = tab[S.src[e]];
    const int d = S.dir[e];
    const int n = S.n[e];
    double sum = 0.0;
    for (int m = 0; m < n; m++) sum += F.E[(d - 1) * F.v.nc + S.si[4 * e + m]];
    tmp[e] = sum * (1.0 / (double)n);
}

__global__ void k_edge_scatter(const DevBlock* tab, SyncDev S, int beg, int end, const double* tmp) {
    const int e = beg + (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= end) return;
    const DevBlock& D = tab[S.dst[e]];
    D.E[(S.dir[e] - 1) * D.v.nc + S.di[e]] = tmp[e];
}

// ------------------------------------------------------------------ reflux records
struct FaceRecDev {
    const int *c, *f, *d, *n;
    const long *fi, *ff;  // coarse face index, fine face indices (4 per record)
    double *own, *acc;    // [NFLUX][nrec]
    const double* sgnh;   // sign / cell size along d (the correction of the adjacent coarse cell)
    double* dU;           // [NCONS][nrec]
};
struct EdgeRecDev {
    const int *c, *f, *e, *n;
    const long *ei, *fe;
    double *own, *acc;
};

__global__ void k_face_own(const DevBlock* tab, FaceRecDev R, int nrec, int lat) {
    const int r = (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= nrec) return;
    const DevBlock& C = tab[R.c[r]];
    if (C.lat != lat) return;
    const int d = R.d[r];
    const double* F = (d == 1) ? C.F1 : ((d == 2) ? C.F2 : C.F3);
    const double dt = C.dscal[0];
    for (int q = 0; q < NFLUX; q++) {
        R.own[(long)q * nrec + r] = dt * F[q * C.v.nc + R.fi[r]];
        R.acc[(long)q * nrec + r] = 0.0;
    }
}

__global__ void k_face_acc(const DevBlock* tab, FaceRecDev R, int nrec, int lat) {
    const int r = (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= nrec) return;
    const DevBlock& Fb = tab[R.f[r]];
    if (Fb.lat != lat) return;
    const int d = R.d[r];
    const double* F = (d == 1) ? Fb.F1 : ((d == 2) ? Fb.F2 : Fb.F3);
    const double dt = Fb.dscal[0];
    const int n = R.n[r];
    for (int q = 0; q < NFLUX; q++) {
        double sum = 0.0;
        for (int m = 0; m < n; m++) sum += F[q * Fb.v.nc + R.ff[4 * r + m]];
        R.acc[(long)q * nrec + r] += dt * (sum * (1.0 / (double)n));
    }
}

__global__ void k_edge_own(const DevBlock* tab, EdgeRecDev R, int nrec, int lat) {
    const int r = (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= nrec) return;
    const DevBlock& C = tab[R.c[r]];
    if (C.lat != lat) return;
    R.own[r] = C.dscal[0] * C.E[(R.e[r] - 1) * C.v.nc + R.ei[r]];
    R.acc[r] = 0.0;
}

__global__ void k_edge_acc(const DevBlock* tab, EdgeRecDev R, int nrec, int lat) {
    const int r = (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= nrec) return;
    const DevBlock& Fb = tab[R.f[r]];
    if (Fb.lat != lat) return;
    const int n = R.n[r];
    double sum = 0.0;
    for (int m = 0; m < n; m++) sum += Fb.E[(R.e[r] - 1) * Fb.v.nc + R.fe[4 * r + m]];
    R.acc[r] += Fb.dscal[0] * (sum * (1.0 / (double)n));
}

// per face record of coarse blocks of level lat: its correction of the adjacent cell
__global__ void k_face_du(const DevBlock* tab, FaceRecDev R, int nrec, int lat) {
    const int r = (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= nrec) return;
    if (tab[R.c[r]].lat != lat) return;
    for (int q = 0; q < NCONS; q++)
        R.dU[(long)q * nrec + r] = R.sgnh[r] * (R.acc[(long)q * nrec + r] - R.own[(long)q * nrec + r]);
}

// the EMF corrections of coarse blocks of level lat, written into their (zeroed) E arrays
__global__ void k_edge_corr(const DevBlock* tab, EdgeRecDev R, int nrec, int lat) {
    const int r = (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= nrec) return;
    const DevBlock& C = tab[R.c[r]];
    if (C.lat != lat) return;
    C.E[(R.e[r] - 1) * C.v.nc + R.ei[r]] = R.acc[r] - R.own[r];
}

__global__ void k_zero_E(const DevBlock* tab, const int* list) {
    const DevBlock& D = tab[list[blockIdx.y]];
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * D.v.nc) return;
    D.E[t] = 0.0;
}

// ------------------------------------------------------------------ period dt and counters
__global__ void k_period_begin(const DevBlock* tab, int nb) {
    const int b = (int)((long)blockIdx.x * blockDim.x + threadIdx.x);
    if (b >= nb) return;
    tab[b].dmax[0] = 0ull;
    for (int q = 0; q < 5; q++) tab[b].dcnt[q] = 0ull;
}

// dtf_out[1] > 0: the caller's fine dt (hamr_grid_set_fine_dt), else the CFL dt of the blocks' rates
__global__ void k_period_dt(const DevBlock* tab, int nb, double cour, double* dtf_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double dtf = 1e300;
    if (dtf_out[1] > 0.0) {
        dtf = dtf_out[1];
    } else {
        for (int b = 0; b < nb; b++) {
            const double rate = __longlong_as_double((long long)tab[b].dmax[0]);
            dtf = fmin(dtf, cour / rate / (double)(1 << tab[b].lat));
        }
    }
    for (int b = 0; b < nb; b++) tab[b].dscal[0] = dtf * (double)(1 << tab[b].lat);
    dtf_out[0] = dtf;
}

// ------------------------------------------------------------------ host-side links
struct HostDomain {
    std::vector<DevBlock> b;
    std::vector<int> bucket;
    AmrDomain A;  // host copy (bucket pointer = host vector)
};

int hfind(const HostDomain& H, const double x[4]) { return find_block(H.A, H.b.data(), x); }

void wrap(const HostDomain& H, double& x, int d, const DevBlock& N) {
    if (!H.A.per[d]) return;
    const double L = H.A.dhi[d] - H.A.dlo[d];
    if (x < N.lo[d] - 1e-9 * L) x += L;
    if (x > N.hi[d] + 1e-9 * L) x -= L;
}

bool finer_than(const DevBlock& A, const DevBlock& C) {
    bool st = false;
    for (int d = 1; d <= 3; d++) {
        if (A.h[d] > C.h[d] * (1 + 1e-9)) return false;
        if (A.h[d] < C.h[d] * (1 - 1e-9)) st = true;
    }
    return st;
}

bool dominates(const HostDomain& H, int a, int c, int e) {
    const DevBlock& A = H.b[a];
    const DevBlock& C = H.b[c];
    if (A.h[e] != C.h[e]) return A.h[e] < C.h[e];
    const double va = A.h[1] * A.h[2] * A.h[3], vc = C.h[1] * C.h[2] * C.h[3];
    if (va != vc) return va < vc;
    return a < c;
}

void blocks_around_edge(const HostDomain& H, int b, const double p[4], int e, std::vector<int>& out) {
    const DevBlock& B = H.b[b];
    const int a1 = (e == 1) ? 2 : 1, a2 = (e == 3) ? 2 : 3;
    out.clear();
    for (int sa = -1; sa <= 1; sa += 2)
        for (int sb = -1; sb <= 1; sb += 2) {
            double x[4] = {0.0, p[1], p[2], p[3]};
            x[a1] += sa * 0.25 * B.h[a1];
            x[a2] += sb * 0.25 * B.h[a2];
            bool outside = false;
            for (int d = 1; d <= 3; d++) {
                if (H.A.per[d]) {
                    const double L = H.A.dhi[d] - H.A.dlo[d];
                    if (x[d] < H.A.dlo[d]) x[d] += L;
                    if (x[d] >= H.A.dhi[d]) x[d] -= L;
                } else if (x[d] < H.A.dlo[d] || x[d] > H.A.dhi[d]) {
                    outside = true;
                }
            }
            if (outside) continue;
            const int n = hfind(H, x);
            if (n >= 0 && std::find(out.begin(), out.end(), n) == out.end()) out.push_back(n);
        }
}

void cover_edge(const HostDomain& H, int n, const double p[4], int e, double he, std::vector<long>& out) {
    const DevBlock& N = H.b[n];
    out.clear();
    int idx[4] = {0, 0, 0, 0};
    for (int d = 1; d <= 3; d++) {
        if (d == e) continue;
        double x = p[d];
        wrap(H, x, d, N);
        idx[d] = (int)llround((x - N.lo[d]) / N.h[d]);
    }
    int cnt = std::max(1, (int)llround(he / N.h[e]));
    double x0 = p[e] - 0.5 * he;
    if (H.A.per[e]) {
        const double L = H.A.dhi[e] - H.A.dlo[e];
        if (x0 < N.lo[e] - 1e-9 * L) x0 += L;
        if (x0 > N.hi[e] - 1e-9 * L) x0 -= L;
    }
    const int i0 = (int)llround((x0 - N.lo[e]) / N.h[e]);
    for (int c = 0; c < cnt; c++) {
        idx[e] = i0 + c;
        out.push_back(pidx(N.v, idx[1], idx[2], idx[3]));
    }
}

void cover_face(const HostDomain& H, int n, const double p[4], int d, const double hb[4], std::vector<long>& out) {
    const DevBlock& N = H.b[n];
    out.clear();
    int i0[4], cnt[4];
    for (int e = 1; e <= 3; e++) {
        double x = p[e];
        wrap(H, x, e, N);
        if (e == d) {
            i0[e] = (int)llround((x - N.lo[e]) / N.h[e]);
            cnt[e] = 1;
        } else {
            cnt[e] = std::max(1, (int)llround(hb[e] / N.h[e]));
            i0[e] = (int)llround((x - 0.5 * hb[e] - N.lo[e]) / N.h[e]);
        }
    }
    for (int c3 = 0; c3 < cnt[3]; c3++)
        for (int c2 = 0; c2 < cnt[2]; c2++)
            for (int c1 = 0; c1 < cnt[1]; c1++) out.push_back(pidx(N.v, i0[1] + c1, i0[2] + c2, i0[3] + c3));
}

struct HSync {
    int dst, dir, src;
    long di;
    std::vector<long> si;
};
struct HFace {
    int c, d, side, i, j, k, f;
    std::vector<long> ff;
};
struct HEdge {
    int c, e, i, j, k, f;
    std::vector<long> fe;
};

}  // namespace

// ------------------------------------------------------------------ AmrImpl
struct AmrImpl {
    PhysArgs ph;
    int nb = 0, Lmax = 0;
    HostDomain H;
    DevBlock* dtab = nullptr;
    int* dbucket = nullptr;
    std::vector<void*> allocs;
    std::vector<std::vector<int>> lev;  // blocks of each level
    std::vector<int*> dlev;             // device copies
    int* dall = nullptr;                // all blocks
    long mw_pad = 0, mw_recon = 0, mw_flux[4] = {0, 0, 0, 0}, mw_edge = 0, mw_cell = 0;
    std::vector<long> lmw_pad, lmw_edge, lmw_cell, lmw_ext;
    std::vector<std::vector<long>> lmw_flux, lmw_recon;
    // synchronisation
    SyncDev fs{}, es{};
    std::vector<int> fs_beg, fs_end, es_beg, es_end;
    double* es_tmp = nullptr;
    int n_fs = 0, n_es = 0;
    // reflux
    FaceRecDev fr{};
    EdgeRecDev er{};
    int n_fr = 0, n_er = 0;
    std::vector<int> rc_beg, rc_end;  // refluxed cells per level: single cells first, then whole SMR groups
    std::vector<int> rc_sgl;          // end of each level's single cells
    std::vector<int> rg_beg, rg_end;  // refluxed SMR groups per level
    int* rg_first = nullptr;          // first list position of each group, relative to its level's rc_beg
    int* rg_w = nullptr;              // its cells
    int* rc_blk = nullptr;
    long* rc_idx = nullptr;
    int* rc_nrec = nullptr;
    int* rc_recs = nullptr;
    double* rc_U = nullptr;
    int n_rc = 0;
    std::vector<std::vector<int>> lev_edgefix;  // blocks of each level with edge corrections
    std::vector<int*> dlev_edgefix;
    std::vector<std::vector<int>> lev_smr;  // blocks of each level with internal-SMR rows
    std::vector<int*> dlev_smr;
    std::vector<long> lmw_smr_emf, lmw_smr_cell;
    double* dtf = nullptr;
    // stored ghost locations (use_maps false: the direct kernels locate on every launch)
    GhostLoc *gloc_cell = nullptr, *gloc_face = nullptr;
    long n_gc = 0, n_gf = 0;
    bool use_maps = false, maps_ok = false;
    std::vector<long> lmw_gc, lmw_gf;  // most ghost cells / faces of a block of each level
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = nullptr;

    template <typename T>
    T* dev(const std::vector<T>& h) {
        T* p = nullptr;
        size_t n = std::max<size_t>(h.size(), 1);
        if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        if (!h.empty()) cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        return p;
    }
    ~AmrImpl() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        for (void* p : allocs) cudaFree(p);
    }
};

namespace {

int build_links(AmrImpl& M, std::vector<HSync>& fsync, std::vector<HSync>& esync, std::vector<HFace>& frec,
                std::vector<HEdge>& erec) {
    const HostDomain& H = M.H;
    for (int b = 0; b < M.nb; b++) {
        const DevBlock& B = H.b[b];
        const int nn[4] = {0, B.v.n1, B.v.n2, B.v.n3};
        for (int fd = 1; fd <= 3; fd++)
            for (int side = 0; side < 2; side++) {
                const int bcv = B.v.bc[2 * (fd - 1) + side];
                if (bcv != HAMR_BC_BLOCK && bcv != HAMR_BC_PERIODIC) continue;
                const int t1 = (fd == 1) ? 2 : 1, t2 = (fd == 3) ? 2 : 3;
                for (int b2 = 0; b2 < nn[t2]; b2++)
                    for (int b1 = 0; b1 < nn[t1]; b1++) {
                        int ii[4];
                        ii[fd] = side ? nn[fd] : 0;
                        ii[t1] = b1;
                        ii[t2] = b2;
                        double p[4] = {0.0, B.lo[1] + (ii[1] + 0.5) * B.h[1], B.lo[2] + (ii[2] + 0.5) * B.h[2],
                                       B.lo[3] + (ii[3] + 0.5) * B.h[3]};
                        p[fd] = side ? B.hi[fd] : B.lo[fd];
                        double q[4] = {0.0, p[1], p[2], p[3]};
                        q[fd] += (side ? 0.25 : -0.25) * B.h[fd];
                        if (H.A.per[fd]) {
                            const double L = H.A.dhi[fd] - H.A.dlo[fd];
                            if (q[fd] < H.A.dlo[fd]) q[fd] += L;
                            if (q[fd] >= H.A.dhi[fd]) q[fd] -= L;
                        }
                        const int n = hfind(H, q);
                        if (n < 0 || n == b) continue;
                        const DevBlock& N = H.b[n];
                        if (!finer_than(N, B) && !(N.lat < B.lat)) continue;
                        const long fi = pidx(B.v, ii[1], ii[2], ii[3]);
                        std::vector<long> cov;
                        cover_face(H, n, p, fd, B.h, cov);
                        if (cov.size() > 4) return -1;
                        if (N.lat == B.lat) {
                            if (!finer_than(N, B)) continue;
                            fsync.push_back({b, fd, n, fi, cov});
                        } else {
                            frec.push_back({b, fd, side, ii[1], ii[2], ii[3], n, cov});
                        }
                    }
            }
        for (int e = 1; e <= 3; e++) {
            const int a1 = (e == 1) ? 2 : 1, a2 = (e == 3) ? 2 : 3;
            for (int k = 0; k <= nn[3]; k++)
                for (int j = 0; j <= nn[2]; j++)
                    for (int i = 0; i <= nn[1]; i++) {
                        const int ii[4] = {0, i, j, k};
                        if (ii[e] >= nn[e]) continue;
                        const bool bnd = (ii[a1] == 0 || ii[a1] == nn[a1] || ii[a2] == 0 || ii[a2] == nn[a2]);
                        if (!bnd) continue;
                        if (e != 2 && ((B.v.bc[2] == HAMR_BC_POLAR && j == 0) || (B.v.bc[3] == HAMR_BC_POLAR && j == nn[2])))
                            continue;
                        double p[4];
                        for (int d = 1; d <= 3; d++) p[d] = B.lo[d] + ii[d] * B.h[d];
                        p[e] += 0.5 * B.h[e];
                        std::vector<int> around;
                        blocks_around_edge(H, b, p, e, around);
                        int gd = b;
                        for (int n : around)
                            if (H.b[n].lat < H.b[gd].lat || (H.b[n].lat == H.b[gd].lat && dominates(H, n, gd, e))) gd = n;
                        int sd = b;
                        for (int n : around)
                            if (H.b[n].lat == B.lat && dominates(H, n, sd, e)) sd = n;
                        const long ei = pidx(B.v, i, j, k);
                        if (sd != b) {
                            HSync r{b, e, sd, ei, {}};
                            cover_edge(H, sd, p, e, B.h[e], r.si);
                            if (r.si.size() > 4) return -1;
                            esync.push_back(r);
                        }
                        if (H.b[gd].lat < B.lat) {
                            HEdge r{b, e, i, j, k, gd, {}};
                            cover_edge(H, gd, p, e, B.h[e], r.fe);
                            if (r.fe.size() > 4) return -1;
                            erec.push_back(r);
                        }
                    }
        }
    }
    return 0;
}

}  // namespace

int amr_create(AmrImpl** out, const hamr_grid_desc& d, const std::vector<BlockView>& views,
               const std::vector<BlockState>& st, const PhysArgs& ph) {
    *out = nullptr;
    AmrImpl* M = new AmrImpl;
    M->ph = ph;
    M->nb = d.nblocks;
    HostDomain& H = M->H;
    H.b.resize(M->nb);
    for (int e = 1; e <= 3; e++) {
        H.A.dlo[e] = 1e300;
        H.A.dhi[e] = -1e300;
        H.A.per[e] = 0;
    }
    double bmin[4] = {0, 1e300, 1e300, 1e300};
    for (int b = 0; b < M->nb; b++) {
        const hamr_block_desc& o = d.blocks[b];
        DevBlock& D = H.b[b];
        std::memset(&D, 0, sizeof(D));
        D.v = views[b];
        const double x0[4] = {0, o.x1min, o.x2min, o.x3min}, hh[4] = {0, o.dx1, o.dx2, o.dx3};
        const int nn[4] = {0, o.n1, o.n2, o.n3};
        for (int e = 1; e <= 3; e++) {
            D.lo[e] = x0[e];
            D.h[e] = hh[e];
            D.hi[e] = x0[e] + nn[e] * hh[e];
            H.A.dlo[e] = std::min(H.A.dlo[e], D.lo[e]);
            H.A.dhi[e] = std::max(H.A.dhi[e], D.hi[e]);
            bmin[e] = std::min(bmin[e], D.hi[e] - D.lo[e]);
            if (o.bc[2 * (e - 1)] == HAMR_BC_PERIODIC) H.A.per[e] = 1;
        }
        if (o.lat < 0 || o.lat > 7) {
            delete M;
            return set_error(HAMR_EINVAL, "block %d: lat must be in 0..7", b);
        }
        D.lat = o.lat;
        M->Lmax = std::max(M->Lmax, o.lat);
        if (ph.smr > 0 && smr_polar(o) && !smr_factors(d, o, &D.v.smr_l2, &D.v.smr_l3)) {
            delete M;
            return set_error(HAMR_EINVAL, "block %d: internal SMR needs cell widths a power of 2 finer", b);
        }
        const BlockState& s = st[b];
        D.P = s.P;
        D.B = s.B;
        D.Ph = s.Ph;
        D.Bh = s.Bh;
        D.QL = s.QL;
        D.QR = s.QR;
        D.P32 = s.P32;
        D.F1 = s.F[0];
        D.F2 = s.F[1];
        D.F3 = s.F[2];
        D.E = s.E;
        D.Un = s.Un;
        D.status = s.status;
        D.dscal = s.dscal;
        D.dmax = s.dmax;
        D.dcnt = s.dcnt;
        void* old = nullptr;
        if (cudaMalloc(&old, sizeof(double) * 11 * views[b].nc) != cudaSuccess) {
            cudaGetLastError();
            delete M;
            return set_error(HAMR_ENOMEM, "allocation of the time-interpolation state of block %d failed", b);
        }
        M->allocs.push_back(old);
        cudaMemset(old, 0, sizeof(double) * 11 * views[b].nc);
        D.Pold = (double*)old;
        D.Bold = D.Pold + 8 * views[b].nc;
    }
    // bucket grid at the smallest block extent; every block must be aligned to it
    for (int e = 1; e <= 3; e++) {
        H.A.bkh[e] = bmin[e];
        H.A.nbk[e] = (int)llround((H.A.dhi[e] - H.A.dlo[e]) / bmin[e]);
    }
    const long nbk = (long)H.A.nbk[1] * H.A.nbk[2] * H.A.nbk[3];
    if (nbk > (1L << 24)) {
        delete M;
        return set_error(HAMR_EINVAL, "block layout too irregular for the bucket lookup");
    }
    H.bucket.assign(nbk, -1);
    for (int b = 0; b < M->nb; b++) {
        const DevBlock& D = H.b[b];
        int lo[4], hi[4];
        for (int e = 1; e <= 3; e++) {
            const double a = (D.lo[e] - H.A.dlo[e]) / H.A.bkh[e], z = (D.hi[e] - H.A.dlo[e]) / H.A.bkh[e];
            lo[e] = (int)llround(a);
            hi[e] = (int)llround(z);
            if (std::fabs(a - lo[e]) > 1e-6 || std::fabs(z - hi[e]) > 1e-6) {
                delete M;
                return set_error(HAMR_EINVAL, "block %d is not aligned to the block grid", b);
            }
        }
        for (int k = lo[3]; k < hi[3]; k++)
            for (int j = lo[2]; j < hi[2]; j++)
                for (int i = lo[1]; i < hi[1]; i++) {
                    int& slot = H.bucket[((long)k * H.A.nbk[2] + j) * H.A.nbk[1] + i];
                    if (slot >= 0) {
                        delete M;
                        return set_error(HAMR_EINVAL, "blocks %d and %d overlap", slot, b);
                    }
                    slot = b;
                }
    }
    for (long q = 0; q < nbk; q++)
        if (H.bucket[q] < 0) {
            delete M;
            return set_error(HAMR_EINVAL, "the blocks leave a hole in the domain");
        }
    H.A.bucket = H.bucket.data();
    H.A.tab = H.b.data();
    H.A.nb = M->nb;

    std::vector<HSync> fsync, esync;
    std::vector<HFace> frec;
    std::vector<HEdge> erec;
    if (build_links(*M, fsync, esync, frec, erec)) {
        delete M;
        return set_error(HAMR_EINVAL, "a face or edge is covered by more than 4 finer faces or edges");
    }
    // every precomputed index must address the block's padded arrays
    {
        auto ok = [&](int b, long i) {
            const BlockView& v = H.b[b].v;
            return b >= 0 && b < M->nb && i >= 0 && i < (long)v.n1p * v.n2p * v.n3p;
        };
        bool good = true;
        for (const HSync& r : fsync) {
            good = good && ok(r.dst, r.di);
            for (long q : r.si) good = good && ok(r.src, q);
        }
        for (const HSync& r : esync) {
            good = good && ok(r.dst, r.di);
            for (long q : r.si) good = good && ok(r.src, q);
        }
        for (const HFace& r : frec) {
            good = good && ok(r.c, pidx(H.b[r.c].v, r.i, r.j, r.k));
            for (long q : r.ff) good = good && ok(r.f, q);
        }
        for (const HEdge& r : erec) {
            good = good && ok(r.c, pidx(H.b[r.c].v, r.i, r.j, r.k));
            for (long q : r.fe) good = good && ok(r.f, q);
        }
        if (!good) {
            delete M;
            return set_error(HAMR_EINVAL, "inconsistent block layout: a link index falls outside its block");
        }
    }
    // sort the synchronisation entries by the level of their destination (stable: keep order)
    auto by_level = [&](std::vector<HSync>& v, std::vector<int>& beg, std::vector<int>& end) {
        std::stable_sort(v.begin(), v.end(), [&](const HSync& a, const HSync& b) { return H.b[a.dst].lat < H.b[b.dst].lat; });
        beg.assign(M->Lmax + 1, 0);
        end.assign(M->Lmax + 1, 0);
        for (int L = 0; L <= M->Lmax; L++) {
            beg[L] = (int)(std::lower_bound(v.begin(), v.end(), L, [&](const HSync& a, int l) { return H.b[a.dst].lat < l; }) - v.begin());
            end[L] = (int)(std::upper_bound(v.begin(), v.end(), L, [&](int l, const HSync& a) { return l < H.b[a.dst].lat; }) - v.begin());
        }
    };
    by_level(fsync, M->fs_beg, M->fs_end);
    by_level(esync, M->es_beg, M->es_end);
    auto sync_dev = [&](const std::vector<HSync>& v, SyncDev& S) {
        std::vector<int> dst, dir, src, n;
        std::vector<long> di, si;
        for (const HSync& r : v) {
            dst.push_back(r.dst);
            dir.push_back(r.dir);
            src.push_back(r.src);
            n.push_back((int)r.si.size());
            di.push_back(r.di);
            for (int m = 0; m < 4; m++) si.push_back(m < (int)r.si.size() ? r.si[m] : 0);
        }
        S.dst = M->dev(dst);
        S.dir = M->dev(dir);
        S.src = M->dev(src);
        S.n = M->dev(n);
        S.di = M->dev(di);
        S.si = M->dev(si);
    };
    sync_dev(fsync, M->fs);
    sync_dev(esync, M->es);
    M->n_fs = (int)fsync.size();
    M->n_es = (int)esync.size();
    M->es_tmp = M->dev(std::vector<double>(std::max<size_t>(esync.size(), 1), 0.0));

    // reflux records
    {
        std::vector<int> c, f, dd, n;
        std::vector<long> fi, ff;
        std::vector<double> sgnh;
        for (const HFace& r : frec) {
            c.push_back(r.c);
            f.push_back(r.f);
            dd.push_back(r.d);
            n.push_back((int)r.ff.size());
            fi.push_back(pidx(H.b[r.c].v, r.i, r.j, r.k));
            for (int m = 0; m < 4; m++) ff.push_back(m < (int)r.ff.size() ? r.ff[m] : 0);
            sgnh.push_back((r.side ? -1.0 : 1.0) / H.b[r.c].h[r.d]);
        }
        M->n_fr = (int)frec.size();
        M->fr.c = M->dev(c);
        M->fr.f = M->dev(f);
        M->fr.d = M->dev(dd);
        M->fr.n = M->dev(n);
        M->fr.fi = M->dev(fi);
        M->fr.ff = M->dev(ff);
        M->fr.sgnh = M->dev(sgnh);
        std::vector<double> z((size_t)NFLUX * std::max(M->n_fr, 1), 0.0);
        M->fr.own = M->dev(z);
        M->fr.acc = M->dev(z);
        M->fr.dU = M->dev(z);
    }
    {
        std::vector<int> c, f, e, n;
        std::vector<long> ei, fe;
        for (const HEdge& r : erec) {
            c.push_back(r.c);
            f.push_back(r.f);
            e.push_back(r.e);
            n.push_back((int)r.fe.size());
            ei.push_back(pidx(H.b[r.c].v, r.i, r.j, r.k));
            for (int m = 0; m < 4; m++) fe.push_back(m < (int)r.fe.size() ? r.fe[m] : 0);
        }
        M->n_er = (int)erec.size();
        M->er.c = M->dev(c);
        M->er.f = M->dev(f);
        M->er.e = M->dev(e);
        M->er.n = M->dev(n);
        M->er.ei = M->dev(ei);
        M->er.fe = M->dev(fe);
        std::vector<double> z(std::max(M->n_er, 1), 0.0);
        M->er.own = M->dev(z);
        M->er.acc = M->dev(z);
    }
    // refluxed cells: the cell next to each face record, and the cells on both
    // sides of every face bounded by a corrected edge; per block, in cell order
    {
        struct RC {
            int blk;
            long idx;
            std::vector<int> recs;
        };
        std::vector<std::vector<RC>> per_block(M->nb);
        auto add_cell = [&](int b, int i, int j, int k, int rec) {
            const DevBlock& B = H.b[b];
            if (i < 0 || j < 0 || k < 0 || i >= B.v.n1 || j >= B.v.n2 || k >= B.v.n3) return;
            const long c = pidx(B.v, i, j, k);
            for (RC& x : per_block[b])
                if (x.idx == c) {
                    if (rec >= 0) x.recs.push_back(rec);
                    return;
                }
            RC x{b, c, {}};
            if (rec >= 0) x.recs.push_back(rec);
            per_block[b].push_back(x);
        };
        for (int r = 0; r < (int)frec.size(); r++) {
            int ii[4] = {0, frec[r].i, frec[r].j, frec[r].k};
            if (frec[r].side == 1) ii[frec[r].d]--;
            add_cell(frec[r].c, ii[1], ii[2], ii[3], r);
        }
        std::vector<char> edgefix(M->nb, 0);
        for (const HEdge& r : erec) {
            edgefix[r.c] = 1;
            const int a1 = (r.e == 1) ? 2 : 1, a2 = (r.e == 3) ? 2 : 3;
            // faces of directions a1 and a2 bounded by the edge, and the cells on both sides of each
            for (int fa : {a1, a2}) {
                const int ob = (fa == a1) ? a2 : a1;  // the face spans the edge's other normal direction
                for (int off = -1; off <= 0; off++) {
                    int face[4] = {0, r.i, r.j, r.k};
                    face[ob] += off;  // the two faces of direction fa touching the edge
                    for (int side = -1; side <= 0; side++) {
                        int cell[4] = {0, face[1], face[2], face[3]};
                        cell[fa] += side;
                        add_cell(r.c, cell[1], cell[2], cell[3], -1);
                    }
                }
            }
        }
        // internal SMR: a group is inverted as one cell, so every cell of a group with a refluxed cell is
        // refluxed
        auto cell_of = [](const BlockView& v, long c, int* i, int* j, int* k) {
            *i = (int)(c % v.n1p) - NG;
            *j = (int)((c / v.n1p) % v.n2p) - NG;
            *k = (int)(c / ((long)v.n1p * v.n2p)) - NG;
        };
        if (ph.smr > 0)
            for (int b = 0; b < M->nb; b++) {
                const BlockView& v = H.b[b].v;
                const size_t n0 = per_block[b].size();
                for (size_t q = 0; q < n0; q++) {
                    int i, j, k;
                    cell_of(v, per_block[b][q].idx, &i, &j, &k);
                    const int w = smr_width(v, ph, j);
                    for (int m = 0; w > 1 && m < w; m++) add_cell(b, i, j, k - k % w + m, -1);
                }
            }
        std::vector<int> blk, nrec, recs, gfirst, gw;
        std::vector<long> idx;
        auto push = [&](const RC& x) {
            blk.push_back(x.blk);
            idx.push_back(x.idx);
            nrec.push_back((int)x.recs.size());
            std::vector<int> rs = x.recs;
            std::sort(rs.begin(), rs.end());
            for (int m = 0; m < 3; m++) recs.push_back(m < (int)rs.size() ? rs[m] : 0);
        };
        M->rc_beg.assign(M->Lmax + 1, 0);
        M->rc_end.assign(M->Lmax + 1, 0);
        M->rc_sgl.assign(M->Lmax + 1, 0);
        M->rg_beg.assign(M->Lmax + 1, 0);
        M->rg_end.assign(M->Lmax + 1, 0);
        for (int L = 0; L <= M->Lmax; L++) {
            M->rc_beg[L] = (int)blk.size();
            for (int b = 0; b < M->nb; b++) {
                if (H.b[b].lat != L) continue;
                std::vector<RC>& v = per_block[b];
                std::sort(v.begin(), v.end(), [](const RC& a, const RC& c) { return a.idx < c.idx; });
                for (const RC& x : v) {
                    if (x.recs.size() > 3) {
                        delete M;
                        return set_error(HAMR_EINVAL, "a refluxed cell with more than 3 corrected faces");
                    }
                    int i, j, k;
                    cell_of(H.b[b].v, x.idx, &i, &j, &k);
                    if (smr_width(H.b[b].v, ph, j) == 1) push(x);
                }
            }
            M->rc_sgl[L] = (int)blk.size();
            M->rg_beg[L] = (int)gfirst.size();
            for (int b = 0; b < M->nb; b++) {
                if (H.b[b].lat != L) continue;
                const BlockView& bv = H.b[b].v;
                for (const RC& x : per_block[b]) {  // sorted by cell: a group's first cell comes first
                    int i, j, k;
                    cell_of(bv, x.idx, &i, &j, &k);
                    const int w = smr_width(bv, ph, j);
                    if (w == 1 || k % w != 0) continue;
                    gfirst.push_back((int)blk.size() - M->rc_beg[L]);
                    gw.push_back(w);
                    for (int m = 0; m < w; m++) {
                        const long c = pidx(bv, i, j, k + m);
                        for (const RC& y : per_block[b])
                            if (y.idx == c) push(y);
                    }
                }
            }
            M->rg_end[L] = (int)gfirst.size();
            M->rc_end[L] = (int)blk.size();
        }
        M->rg_first = M->dev(gfirst);
        M->rg_w = M->dev(gw);
        M->n_rc = (int)blk.size();
        M->rc_blk = M->dev(blk);
        M->rc_idx = M->dev(idx);
        M->rc_nrec = M->dev(nrec);
        M->rc_recs = M->dev(recs);
        M->rc_U = M->dev(std::vector<double>((size_t)NCONS * std::max(M->n_rc, 1), 0.0));
        M->lev_edgefix.assign(M->Lmax + 1, {});
        for (int b = 0; b < M->nb; b++)
            if (edgefix[b]) M->lev_edgefix[H.b[b].lat].push_back(b);
        for (int L = 0; L <= M->Lmax; L++) M->dlev_edgefix.push_back(M->dev(M->lev_edgefix[L]));
    }
    // device tables
    for (int b = 0; b < M->nb; b++) {
        const BlockView& v = H.b[b].v;
        // dscal[1] = 1 (unit time factor of the EMF-correction curl)
        const double one = 1.0;
        cudaMemcpy(H.b[b].dscal + 1, &one, sizeof(double), cudaMemcpyHostToDevice);
        (void)v;
    }
    // ghost lists in padded order: (t, receiving block) now, the locations on the device below
    std::vector<GhostLoc> gcell, gface;
    for (int b = 0; b < M->nb; b++) {
        DevBlock& D = H.b[b];
        const BlockView& v = D.v;
        const int nn[4] = {0, v.n1, v.n2, v.n3};
        D.gofs_cell = (long)gcell.size();
        for (int k = 0; k < v.n3p; k++)
            for (int j = 0; j < v.n2p; j++)
                for (int i = 0; i < v.n1p; i++) {
                    const int ii[4] = {0, i - NG, j - NG, k - NG};
                    bool ghost = false;
                    for (int e = 1; e <= 3; e++) ghost = ghost || ii[e] < 0 || ii[e] >= nn[e];
                    if (ghost) gcell.push_back({(int)(((long)k * v.n2p + j) * v.n1p + i), b, 0, 0u});
                }
        D.ng_cell = (int)((long)gcell.size() - D.gofs_cell);
        D.gofs_face = (long)gface.size();
        for (int fd = 1; fd <= 3; fd++)
            for (int k = 0; k < v.n3p; k++)
                for (int j = 0; j < v.n2p; j++)
                    for (int i = 0; i < v.n1p; i++) {
                        const int ii[4] = {0, i - NG, j - NG, k - NG};
                        bool ghost = false;
                        for (int e = 1; e <= 3; e++)
                            ghost = ghost || ii[e] < 0 || ii[e] > nn[e] || (e != fd && ii[e] == nn[e]);
                        if (ghost)
                            gface.push_back({(int)(((long)k * v.n2p + j) * v.n1p + i), b, 0, (unsigned)fd << 28});
                    }
        D.ng_face = (int)((long)gface.size() - D.gofs_face);
    }
    M->n_gc = (long)gcell.size();
    M->n_gf = (long)gface.size();
    M->gloc_cell = M->dev(gcell);
    M->gloc_face = M->dev(gface);
    if (!M->gloc_cell || !M->gloc_face) {
        cudaGetLastError();
        delete M;
        return set_error(HAMR_ENOMEM, "allocation of the ghost locations failed");
    }
    M->lmw_gc.assign(M->Lmax + 1, 0);
    M->lmw_gf.assign(M->Lmax + 1, 0);
    for (int b = 0; b < M->nb; b++) {
        M->lmw_gc[H.b[b].lat] = std::max(M->lmw_gc[H.b[b].lat], (long)H.b[b].ng_cell);
        M->lmw_gf[H.b[b].lat] = std::max(M->lmw_gf[H.b[b].lat], (long)H.b[b].ng_face);
    }
    M->dtab = M->dev(H.b);
    M->dbucket = M->dev(H.bucket);
    M->lev.assign(M->Lmax + 1, {});
    std::vector<int> all;
    for (int b = 0; b < M->nb; b++) {
        M->lev[H.b[b].lat].push_back(b);
        all.push_back(b);
    }
    for (int L = 0; L <= M->Lmax; L++) M->dlev.push_back(M->dev(M->lev[L]));
    M->dall = M->dev(all);
    M->lev_smr.assign(M->Lmax + 1, {});
    M->lmw_smr_emf.assign(M->Lmax + 1, 0);
    M->lmw_smr_cell.assign(M->Lmax + 1, 0);
    for (int b = 0; b < M->nb; b++) {
        const long nf = smr_emf_threads(H.b[b].v, ph), ncl = smr_cell_threads(H.b[b].v, ph);
        if (!smr_polar(d.blocks[b]) || nf == 0) continue;
        const int L = H.b[b].lat;
        M->lev_smr[L].push_back(b);
        M->lmw_smr_emf[L] = std::max(M->lmw_smr_emf[L], nf);
        M->lmw_smr_cell[L] = std::max(M->lmw_smr_cell[L], ncl);
    }
    for (int L = 0; L <= M->Lmax; L++) M->dlev_smr.push_back(M->dev(M->lev_smr[L]));
    M->lmw_pad.assign(M->Lmax + 1, 0);
    M->lmw_recon.assign(M->Lmax + 1, std::vector<long>(4, 0));
    M->lmw_edge.assign(M->Lmax + 1, 0);
    M->lmw_cell.assign(M->Lmax + 1, 0);
    M->lmw_ext.assign(M->Lmax + 1, 0);
    M->lmw_flux.assign(M->Lmax + 1, std::vector<long>(4, 0));
    for (int b = 0; b < M->nb; b++) {
        const BlockView& v = H.b[b].v;
        const int L = H.b[b].lat;
        const long pad = (long)v.n1p * v.n2p * v.n3p;
        const long edg = (long)(v.n1 + 1) * (v.n2 + 1) * (v.n3 + 1);
        const long cel = (long)v.n1 * v.n2 * v.n3;
        M->lmw_pad[L] = std::max(M->lmw_pad[L], pad);
        for (int dir = 1; dir <= 3; dir++)
            M->lmw_recon[L][dir] =
                std::max(M->lmw_recon[L][dir], recon_threads(v, dir, ph.mixed, ph.recon_seg, ph.recon_x1_sweep));
        M->lmw_edge[L] = std::max(M->lmw_edge[L], edg);
        M->lmw_cell[L] = std::max(M->lmw_cell[L], cel);
        M->lmw_ext[L] = std::max(M->lmw_ext[L], (long)(v.n1 + 2) * (v.n2 + 2) * (v.n3 + 2));
        M->lmw_flux[L][1] = std::max(M->lmw_flux[L][1], (long)(v.n1 + 1) * (v.n2 + 2) * (v.n3 + 2));
        M->lmw_flux[L][2] = std::max(M->lmw_flux[L][2], (long)(v.n1 + 2) * (v.n2 + 1) * (v.n3 + 2));
        M->lmw_flux[L][3] = std::max(M->lmw_flux[L][3], (long)(v.n1 + 2) * (v.n2 + 2) * (v.n3 + 1));
        M->mw_pad = std::max(M->mw_pad, pad);
        M->mw_cell = std::max(M->mw_cell, cel);
    }
    M->dtf = M->dev(std::vector<double>(4, 0.0));
    H.A.tab = M->dtab;
    H.A.bucket = M->dbucket;
    {
        int* bad = M->dev(std::vector<int>(1, 0));
        if (M->n_gc) k_ghost_cells_locate<<<nb_(M->n_gc), BSA>>>(H.A, M->gloc_cell, M->n_gc, bad);
        if (M->n_gf) k_ghost_faces_locate<<<nb_(M->n_gf), BSA>>>(H.A, M->gloc_face, M->n_gf, bad);
        int hbad = 1;
        if (cudaGetLastError() == cudaSuccess && cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
            M->maps_ok = M->use_maps = (hbad == 0);
    }
    if (cudaStreamCreateWithFlags(&M->cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete M;
        return set_error(HAMR_ECUDA, "stream creation failed");
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete M;
        return set_error(HAMR_ECUDA, "multi-block set-up failed: %s", cudaGetErrorString(e));
    }
    // host-side lookups must keep host pointers
    *out = M;
    return HAMR_OK;
}

void amr_destroy(AmrImpl* M) { delete M; }

int amr_after_load(AmrImpl* M, int b, cudaStream_t s) {
    // no history yet: the previous state is the loaded one
    const DevBlock& D = M->H.b[b];
    cudaError_t e = cudaMemcpyAsync(D.Pold, D.P, sizeof(double) * 8 * D.v.nc, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(D.Bold, D.B, sizeof(double) * 3 * D.v.nc, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_error(HAMR_ECUDA, "state copy failed: %s", cudaGetErrorString(e));
    return HAMR_OK;
}

namespace {

#define AM_TRY(call)                                                                                           \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess) return set_error(HAMR_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int group_step(AmrImpl& M, int L, int s, cudaStream_t cs) {
    const int nl = (int)M.lev[L].size();
    const int* list = M.dlev[L];
    const DevBlock* tab = M.dtab;
    const PhysArgs& ph = M.ph;
    AM_TRY(launch_save_old_batch(tab, list, nl, M.lmw_pad[L], cs));
    for (int sigma = 0; sigma < 2; sigma++) {
        if (M.use_maps) {
            if (M.lmw_gc[L])
                k_ghost_cells_mapped<<<dim3(nb_(M.lmw_gc[L]), nl), BSA, 0, cs>>>(M.H.A, list, sigma, s, M.gloc_cell);
            if (M.lmw_gf[L])
                k_ghost_faces_mapped<<<dim3(nb_(M.lmw_gf[L]), nl), BSA, 0, cs>>>(M.H.A, list, sigma, s, M.gloc_face);
        } else {
            k_ghost_cells<<<dim3(nb_(M.lmw_pad[L]), nl), BSA, 0, cs>>>(M.H.A, list, sigma, s);
            k_ghost_faces<<<dim3(nb_(3 * M.lmw_pad[L]), nl), BSA, 0, cs>>>(M.H.A, list, sigma, s);
        }
        AM_TRY(cudaGetLastError());
        if (ph.mixed) AM_TRY(launch_to_f32_batch(tab, list, nl, M.lmw_pad[L], sigma, cs));
        AM_TRY(launch_kappa_batch(tab, list, nl, M.lmw_pad[L], ph, sigma, cs));
        for (int dir = 1; dir <= 3; dir++) {
            if (ph.flatten) AM_TRY(launch_flatten_batch(tab, list, nl, M.lmw_ext[L], ph, dir, sigma, cs));
            AM_TRY(launch_recon_batch(tab, list, nl, M.lmw_recon[L][dir], ph, dir, sigma, cs));
            AM_TRY(launch_flux_batch(tab, list, nl, M.lmw_flux[L][dir], ph, dir, sigma, cs));
        }
        const int fb = M.fs_beg[L], fe = M.fs_end[L];
        if (fe > fb) k_flux_sync<<<nb_(fe - fb), BSA, 0, cs>>>(tab, M.fs, fb, fe, ph.flux32);
        AM_TRY(launch_emf_batch(tab, list, nl, M.lmw_edge[L], ph.mixed ? (ph.flux32 ? 2 : 1) : 0, ph.emf,
                                M.lmw_ext[L], sigma, cs));
        const int eb = M.es_beg[L], ee = M.es_end[L];
        if (ee > eb) {
            k_edge_gather<<<nb_(ee - eb), BSA, 0, cs>>>(tab, M.es, eb, ee, M.es_tmp);
            k_edge_scatter<<<nb_(ee - eb), BSA, 0, cs>>>(tab, M.es, eb, ee, M.es_tmp);
        }
        AM_TRY(cudaGetLastError());
        // internal SMR: each block's EMFs as its groups' after the exchange
        const int ns = (int)M.lev_smr[L].size();
        if (ns) AM_TRY(launch_smr_emf_batch(tab, M.dlev_smr[L], ns, M.lmw_smr_emf[L], ph, cs));
        if (sigma == 1) {
            if (M.n_fr) {
                k_face_own<<<nb_(M.n_fr), BSA, 0, cs>>>(tab, M.fr, M.n_fr, L);
                k_face_acc<<<nb_(M.n_fr), BSA, 0, cs>>>(tab, M.fr, M.n_fr, L);
            }
            if (M.n_er) {
                k_edge_own<<<nb_(M.n_er), BSA, 0, cs>>>(tab, M.er, M.n_er, L);
                k_edge_acc<<<nb_(M.n_er), BSA, 0, cs>>>(tab, M.er, M.n_er, L);
            }
            AM_TRY(cudaGetLastError());
        }
        AM_TRY(launch_ct_batch(tab, list, nl, M.lmw_edge[L], sigma, cs));
        AM_TRY(launch_update_batch(tab, list, nl, M.lmw_cell[L], ph, sigma, cs));
        if (ns) AM_TRY(launch_smr_cells_batch(tab, M.dlev_smr[L], ns, M.lmw_smr_cell[L], ph, sigma, cs));
    }
    return HAMR_OK;
}

int reflux_level(AmrImpl& M, int L, cudaStream_t cs) {
    const int cb = M.rc_beg[L], ce = M.rc_end[L];
    const int ne = (int)M.lev_edgefix[L].size();
    if (ce == cb && ne == 0) return HAMR_OK;
    const DevBlock* tab = M.dtab;
    if (M.n_fr) k_face_du<<<nb_(M.n_fr), BSA, 0, cs>>>(tab, M.fr, M.n_fr, L);
    AM_TRY(cudaGetLastError());
    AM_TRY(launch_reflux_u0(tab, ce - cb, M.rc_blk + cb, M.rc_idx + cb, M.rc_nrec + cb, M.rc_recs + 3 * cb, M.fr.dU,
                            std::max(M.n_fr, 1), M.rc_U, M.ph, cs));
    if (ne) {
        k_zero_E<<<dim3(nb_(3 * (M.mw_pad + 256)), ne), BSA, 0, cs>>>(tab, M.dlev_edgefix[L]);
        k_edge_corr<<<nb_(M.n_er), BSA, 0, cs>>>(tab, M.er, M.n_er, L);
        AM_TRY(cudaGetLastError());
        long mw = 0;
        for (int b : M.lev_edgefix[L]) {
            const BlockView& v = M.H.b[b].v;
            mw = std::max(mw, (long)(v.n1 + 1) * (v.n2 + 1) * (v.n3 + 1));
        }
        AM_TRY(launch_ct_batch(tab, M.dlev_edgefix[L], ne, mw, 2, cs));
    }
    const int cg = M.rc_sgl[L];
    AM_TRY(launch_reflux_cells(tab, cg - cb, M.rc_blk + cb, M.rc_idx + cb, M.rc_U, ce - cb, M.ph, cs));
    const int gb = M.rg_beg[L], ge = M.rg_end[L];
    AM_TRY(launch_reflux_groups(tab, ge - gb, M.rg_first + gb, M.rg_w + gb, M.rc_blk + cb, M.rc_idx + cb, M.rc_U,
                                ce - cb, M.ph, cs));
    return HAMR_OK;
}

int issue_period(AmrImpl& M, cudaStream_t cs) {
    const DevBlock* tab = M.dtab;
    k_period_begin<<<nb_(M.nb), BSA, 0, cs>>>(tab, M.nb);
    AM_TRY(launch_dt_reduce_batch(tab, M.dall, M.nb, M.mw_cell, M.ph, cs));
    k_period_dt<<<1, 32, 0, cs>>>(tab, M.nb, M.ph.cour, M.dtf);
    AM_TRY(cudaGetLastError());
    const int S = 1 << M.Lmax;
    for (int s = 0; s < S; s++) {
        for (int L = M.Lmax; L >= 0; L--) {
            if (s % (1 << L) != 0 || M.lev[L].empty()) continue;
            int rc = group_step(M, L, s, cs);
            if (rc) return rc;
        }
        for (int L = 0; L <= M.Lmax; L++) {
            if ((s + 1) % (1 << L) != 0) continue;
            int rc = reflux_level(M, L, cs);
            if (rc) return rc;
        }
    }
    return HAMR_OK;
}

}  // namespace

int amr_period(AmrImpl* M, cudaStream_t s, int nperiods, bool use_graph) {
    if (!use_graph) {
        for (int p = 0; p < nperiods; p++) {
            int rc = issue_period(*M, s);
            if (rc) return rc;
        }
        return HAMR_OK;
    }
    if (!M->exec) {
        AM_TRY(cudaStreamBeginCapture(M->cap, cudaStreamCaptureModeThreadLocal));
        int rc = issue_period(*M, M->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(M->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return set_error(HAMR_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        M->graph = g;
        AM_TRY(cudaGraphInstantiate(&M->exec, g, 0));
    }
    for (int p = 0; p < nperiods; p++) AM_TRY(cudaGraphLaunch(M->exec, s));
    return HAMR_OK;
}

int amr_set_phys(AmrImpl* M, const PhysArgs& ph) {
    M->ph = ph;  // the captured period bakes the launch arguments: capture again
    for (int L = 0; L <= M->Lmax; L++)
        for (int dir = 1; dir <= 3; dir++) {
            long mw = 0;
            for (int b : M->lev[L])
                mw = std::max(mw, recon_threads(M->H.b[b].v, dir, ph.mixed, ph.recon_seg, ph.recon_x1_sweep));
            M->lmw_recon[L][dir] = mw;
        }
    if (M->exec) cudaGraphExecDestroy(M->exec);
    if (M->graph) cudaGraphDestroy(M->graph);
    M->exec = nullptr;
    M->graph = nullptr;
    return HAMR_OK;
}

// Time (ms, summed over levels) of one kernel group of the batched step on the
// current state, predictor stage: 0 reconstruction, 1 face fluxes, 2 cell
// update. Writes only scratch (edge values, fluxes, the midpoint state, the
// U^n cache, counters and status bits, which the next period resets).
int amr_time_group(AmrImpl* M, const PhysArgs& ph, int which, cudaStream_t cs, float* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    AM_TRY(cudaEventCreate(&a));
    AM_TRY(cudaEventCreate(&b));
    float total = 0.0f;
    const DevBlock* tab = M->dtab;
    int rc = HAMR_OK;
    for (int L = 0; L <= M->Lmax && rc == HAMR_OK; L++) {
        const int nl = (int)M->lev[L].size();
        if (!nl) continue;
        const int* list = M->dlev[L];
        long mwr[4];
        for (int dir = 1; dir <= 3; dir++) {
            mwr[dir] = 0;
            for (int bb : M->lev[L])
                mwr[dir] = std::max(mwr[dir], recon_threads(M->H.b[bb].v, dir, ph.mixed, ph.recon_seg,
                                                            ph.recon_x1_sweep));
        }
        auto timed = [&](auto launch) {
            cudaEventRecord(a, cs);
            cudaError_t e = launch();
            cudaEventRecord(b, cs);
            if (e != cudaSuccess) return set_error(HAMR_ECUDA, "launch failed: %s", cudaGetErrorString(e));
            e = cudaEventSynchronize(b);
            if (e != cudaSuccess) return set_error(HAMR_ECUDA, "timing failed: %s", cudaGetErrorString(e));
            float t = 0.0f;
            cudaEventElapsedTime(&t, a, b);
            total += t;
            return (int)HAMR_OK;
        };
        if (ph.mixed) {
            cudaError_t e = launch_to_f32_batch(tab, list, nl, M->lmw_pad[L], 0, cs);
            if (e != cudaSuccess) rc = set_error(HAMR_ECUDA, "launch failed: %s", cudaGetErrorString(e));
        }
        if (rc == HAMR_OK) {
            auto kap = [&]() { return launch_kappa_batch(tab, list, nl, M->lmw_pad[L], ph, 0, cs); };
            if (which == 0) {
                rc = timed(kap);
            } else {
                cudaError_t e = kap();
                if (e != cudaSuccess) rc = set_error(HAMR_ECUDA, "launch failed: %s", cudaGetErrorString(e));
            }
        }
        for (int dir = 1; dir <= 3 && rc == HAMR_OK; dir++) {
            auto rec = [&]() {
                cudaError_t e = ph.flatten ? launch_flatten_batch(tab, list, nl, M->lmw_ext[L], ph, dir, 0, cs)
                                           : cudaSuccess;
                return e == cudaSuccess ? launch_recon_batch(tab, list, nl, mwr[dir], ph, dir, 0, cs) : e;
            };
            auto flx = [&]() { return launch_flux_batch(tab, list, nl, M->lmw_flux[L][dir], ph, dir, 0, cs); };
            if (which == 0) {
                rc = timed(rec);
            } else {
                cudaError_t e = rec();
                if (e == cudaSuccess && which == 1) rc = timed(flx);
                else if (e == cudaSuccess) e = flx();
                if (e != cudaSuccess) rc = set_error(HAMR_ECUDA, "launch failed: %s", cudaGetErrorString(e));
            }
        }
        if (rc == HAMR_OK && which == 2)
            rc = timed([&]() { return launch_update_batch(tab, list, nl, M->lmw_cell[L], ph, 0, cs); });
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = total;
    return rc;
}

int amr_fill(AmrImpl* M, cudaStream_t s) {
    // every block at the same time: the stage-0 sources of substep 0 are the current states
    for (int L = 0; L <= M->Lmax; L++) {
        const int nl = (int)M->lev[L].size();
        if (!nl) continue;
        if (M->use_maps) {
            if (M->lmw_gc[L])
                k_ghost_cells_mapped<<<dim3(nb_(M->lmw_gc[L]), nl), BSA, 0, s>>>(M->H.A, M->dlev[L], 0, 0, M->gloc_cell);
            if (M->lmw_gf[L])
                k_ghost_faces_mapped<<<dim3(nb_(M->lmw_gf[L]), nl), BSA, 0, s>>>(M->H.A, M->dlev[L], 0, 0, M->gloc_face);
        } else {
            k_ghost_cells<<<dim3(nb_(M->lmw_pad[L]), nl), BSA, 0, s>>>(M->H.A, M->dlev[L], 0, 0);
            k_ghost_faces<<<dim3(nb_(3 * M->lmw_pad[L]), nl), BSA, 0, s>>>(M->H.A, M->dlev[L], 0, 0);
        }
    }
    AM_TRY(cudaGetLastError());
    return HAMR_OK;
}

int amr_regrid_fill(const AmrImpl* old, AmrImpl* M, cudaStream_t s) {
    long maxc = 1, maxf = 1;
    for (int b = 0; b < M->nb; b++) {
        const BlockView& v = M->H.b[b].v;
        maxc = std::max(maxc, (long)v.n1 * v.n2 * v.n3);
        maxf = std::max(maxf, (long)(v.n1 + 1) * (v.n2 + 1) * (v.n3 + 1));
    }
    k_regrid_cells<<<dim3(nb_(maxc), M->nb), BSA, 0, s>>>(old->H.A, M->dtab);
    k_regrid_faces<<<dim3(nb_(3 * maxf), M->nb), BSA, 0, s>>>(old->H.A, M->dtab);
    AM_TRY(cudaGetLastError());
    for (int b = 0; b < M->nb; b++) {
        const DevBlock& D = M->H.b[b];
        AM_TRY(launch_centre_b(D.v, D.P, D.B, s));
        int rc = amr_after_load(M, b, s);
        if (rc) return rc;
    }
    return amr_fill(M, s);
}

int amr_set_ghost_maps(AmrImpl* M, int on, int* was) {
    if (was) *was = M->use_maps ? 1 : 0;
    if (on && !M->maps_ok) return set_error(HAMR_EINVAL, "this tree's ghost footprints do not fit the stored form");
    const bool u = on != 0;
    if (u != M->use_maps) {  // the captured period holds the other kernels: capture again
        M->use_maps = u;
        if (M->exec) cudaGraphExecDestroy(M->exec);
        if (M->graph) cudaGraphDestroy(M->graph);
        M->exec = nullptr;
        M->graph = nullptr;
    }
    return HAMR_OK;
}

int amr_set_fine_dt(AmrImpl* M, double dt) {
    const double v = dt > 0.0 ? dt : 0.0;
    AM_TRY(cudaMemcpy(M->dtf + 1, &v, sizeof(double), cudaMemcpyHostToDevice));
    return HAMR_OK;
}

int amr_info(const AmrImpl* M, int* lmax, double* dtf_host) {
    *lmax = M->Lmax;
    if (dtf_host) {
        cudaError_t e = cudaMemcpy(dtf_host, M->dtf, sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return set_error(HAMR_ECUDA, "dt read failed: %s", cudaGetErrorString(e));
    }
    return HAMR_OK;
}

int amr_links(const AmrImpl* M, int* counts) {
    counts[0] = M->n_fs;
    counts[1] = M->n_es;
    counts[2] = M->n_fr;
    counts[3] = M->n_er;
    counts[4] = M->n_rc;
    return HAMR_OK;
}

}  // namespace hamr
