// tree.cu -- host-side block-tree adaptation (Sec. 3.2, 3.3.1): per-block target
// levels to a block tree that obeys the paper's nesting rule (a block's face and
// edge neighbours have cells at most a factor 2 wider or narrower in every
// direction), ready for hamr_grid_regrid. Blocks away from a polar axis split
// into 8 octants; blocks touching a polar axis split 6-way: the x2 half at the
// axis into 2 children that keep the parent's x3 cells (halved in x1 and x2),
// the other half into 4 children halved in all three directions. A call moves
// each region by at most one level toward its target (the regrid prolongs and
// restricts by factors of 2); repeat until the tree is stable.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "hamr_internal.h"

namespace {

constexpr int MAX_LEVEL = 10;
constexpr long MAX_UNITS = 1L << 26;  // finest-level block slots of the domain

// A block of the tree: level l in x1 and x2, level lp in x3 (lp < l below a 6-way split on the axis),
// index c[d] on its level's lattice (c[2] on the x3 lattice of level lp), and its base block's cells.
struct Blk {
    int l, lp;
    long c[3];
};

struct Tree {
    int nb[3];      // base blocks per direction
    int Lf;         // finest level
    long U[3];      // finest-level block slots per direction
    bool per[3];
    bool axis[2];   // x2 lower / upper domain face is a polar axis
    std::vector<int8_t> req;  // required level per finest slot
    long idx(long x, long y, long z) const { return (z * U[1] + y) * U[0] + x; }
    long span(int l) const { return 1L << (Lf - l); }
    // largest requirement over the slots of a block
    int max_req(const Blk& b) const {
        const long s = span(b.l), sp = span(b.lp);
        int m = 0;
        for (long z = b.c[2] * sp; z < (b.c[2] + 1) * sp; z++)
            for (long y = b.c[1] * s; y < (b.c[1] + 1) * s; y++)
                for (long x = b.c[0] * s; x < (b.c[0] + 1) * s; x++) m = std::max<int>(m, req[idx(x, y, z)]);
        return m;
    }
    void raise(const Blk& b, int level) {
        const long s = span(b.l), sp = span(b.lp);
        for (long z = b.c[2] * sp; z < (b.c[2] + 1) * sp; z++)
            for (long y = b.c[1] * s; y < (b.c[1] + 1) * s; y++)
                for (long x = b.c[0] * s; x < (b.c[0] + 1) * s; x++) {
                    int8_t& r = req[idx(x, y, z)];
                    if (r < level) r = (int8_t)level;
                }
    }
    // the block touches a polar axis: its x2 side at a domain x2 face that is an axis
    int on_axis(const Blk& b) const {
        const long nl = (long)nb[1] << b.l;
        if (axis[0] && b.c[1] == 0) return 1;         // the axis on its lower x2 side
        if (axis[1] && b.c[1] == nl - 1) return 2;    // on its upper x2 side
        return 0;
    }
};

// leaves of a block: split while a slot needs more (6-way on an axis, else 8-way)
void leaves_of(const Tree& T, const Blk& b, std::vector<Blk>& out) {
    if (b.l < T.Lf && T.max_req(b) > b.l) {
        const int ax = T.on_axis(b);
        for (int jc = 0; jc < 2; jc++)
            for (int ic = 0; ic < 2; ic++) {
                const bool axis_half = (ax == 1 && jc == 0) || (ax == 2 && jc == 1);
                if (axis_half) {
                    Blk ch{b.l + 1, b.lp, {2 * b.c[0] + ic, 2 * b.c[1] + jc, b.c[2]}};
                    leaves_of(T, ch, out);
                } else {
                    for (int kc = 0; kc < 2; kc++) {
                        Blk ch{b.l + 1, b.lp + 1, {2 * b.c[0] + ic, 2 * b.c[1] + jc, 2 * b.c[2] + kc}};
                        leaves_of(T, ch, out);
                    }
                }
            }
        return;
    }
    out.push_back(b);
}

std::vector<Blk> all_leaves(const Tree& T) {
    std::vector<Blk> out;
    for (long kb = 0; kb < T.nb[2]; kb++)
        for (long jb = 0; jb < T.nb[1]; jb++)
            for (long ib = 0; ib < T.nb[0]; ib++) leaves_of(T, Blk{0, 0, {ib, jb, kb}}, out);
    return out;
}

// extent of a block on the finest slot lattice: [lo, hi) per direction
void slot_box(const Tree& T, const Blk& b, long lo[3], long hi[3]) {
    const long s = T.span(b.l), sp = T.span(b.lp);
    for (int d = 0; d < 3; d++) {
        const long w = (d == 2) ? sp : s;
        lo[d] = b.c[d] * w;
        hi[d] = lo[d] + w;
    }
}

// contact of two slot boxes along one direction (with the period): 2 overlap, 1 touch, 0 apart
int contact(long alo, long ahi, long blo, long bhi, long U, bool per) {
    int best = 0;
    const long shifts[3] = {0, U, -U};
    for (int q = 0; q < (per ? 3 : 1); q++) {
        const long lo = std::max(alo, blo + shifts[q]), hi = std::min(ahi, bhi + shifts[q]);
        if (hi > lo) return 2;
        if (hi == lo) best = 1;
    }
    return best;
}

}  // namespace

namespace {

int adapt(const hamr_block_desc* cur, int n, const int* target, const double dlo[3], const double base_ext[3],
          const int periodic[3], const int axis[2], hamr_block_desc* out, int cap, int* nout) {
    using hamr::set_error;
    if (!cur || n < 1 || !target || !dlo || !base_ext || !periodic || !nout)
        return set_error(HAMR_EINVAL, "hamr_tree_adapt: NULL argument or n < 1");
    *nout = 0;
    Tree T;
    T.Lf = 0;
    T.axis[0] = axis && axis[0];
    T.axis[1] = axis && axis[1];
    double hi[3] = {dlo[0], dlo[1], dlo[2]};
    std::vector<Blk> in(n);
    int dbc[6] = {HAMR_BC_OUTFLOW, HAMR_BC_OUTFLOW, HAMR_BC_OUTFLOW, HAMR_BC_OUTFLOW, HAMR_BC_OUTFLOW,
                  HAMR_BC_OUTFLOW};
    for (int b = 0; b < n; b++) {
        const hamr_block_desc& B = cur[b];
        const int nn[3] = {B.n1, B.n2, B.n3};
        const double x0[3] = {B.x1min, B.x2min, B.x3min}, h[3] = {B.dx1, B.dx2, B.dx3};
        int lev[3];
        for (int d = 0; d < 3; d++) {
            if (nn[d] < 1) return set_error(HAMR_EINVAL, "block %d: cell counts must be positive", b);
            const double ext = nn[d] * h[d];
            const int l = (int)std::lround(std::log2(base_ext[d] / ext));
            if (l < 0 || l > MAX_LEVEL || std::fabs(std::ldexp(ext, l) - base_ext[d]) > 1e-9 * base_ext[d])
                return set_error(HAMR_EINVAL, "block %d: extent is not base_ext / 2^L (L <= %d)", b, MAX_LEVEL);
            lev[d] = l;
            const double c = (x0[d] - dlo[d]) / ext;
            in[b].c[d] = std::lround(c);
            if (std::fabs(c - (double)in[b].c[d]) > 1e-6 || in[b].c[d] < 0)
                return set_error(HAMR_EINVAL, "block %d: not on the level-%d block lattice", b, l);
            hi[d] = std::max(hi[d], x0[d] + ext);
            if (std::fabs(x0[d] - dlo[d]) <= 1e-9 * base_ext[d]) dbc[2 * d] = B.bc[2 * d];
        }
        if (lev[0] != lev[1]) return set_error(HAMR_EINVAL, "block %d: levels differ between x1 and x2", b);
        if (lev[2] > lev[0]) return set_error(HAMR_EINVAL, "block %d: finer in x3 than in x1 and x2", b);
        in[b].l = lev[0];
        in[b].lp = lev[2];
        T.Lf = std::max(T.Lf, lev[0]);
        if (target[b] > MAX_LEVEL) return set_error(HAMR_EINVAL, "block %d: target level above %d", b, MAX_LEVEL);
        T.Lf = std::max(T.Lf, std::min(std::max(target[b], 0), MAX_LEVEL));
    }
    long units = 1;
    for (int d = 0; d < 3; d++) {
        T.nb[d] = (int)std::lround((hi[d] - dlo[d]) / base_ext[d]);
        if (T.nb[d] < 1 || std::fabs(T.nb[d] * base_ext[d] - (hi[d] - dlo[d])) > 1e-9 * base_ext[d] * T.nb[d])
            return set_error(HAMR_EINVAL, "the blocks do not span whole base blocks along direction %d", d + 1);
        T.U[d] = (long)T.nb[d] << T.Lf;
        T.per[d] = periodic[d] != 0;
        units *= T.U[d];
        if (units > MAX_UNITS) return set_error(HAMR_EINVAL, "tree too fine: more than %ld finest block slots", MAX_UNITS);
    }
    // the upper domain faces' bc; each base block's cell counts (its descendants keep them)
    std::vector<int> bcells((size_t)3 * T.nb[0] * T.nb[1] * T.nb[2], 0);
    for (int b = 0; b < n; b++) {
        const hamr_block_desc& B = cur[b];
        const double x0[3] = {B.x1min, B.x2min, B.x3min}, h[3] = {B.dx1, B.dx2, B.dx3};
        const int nn[3] = {B.n1, B.n2, B.n3};
        for (int d = 0; d < 3; d++)
            if (std::fabs(x0[d] + nn[d] * h[d] - hi[d]) <= 1e-9 * base_ext[d]) dbc[2 * d + 1] = B.bc[2 * d + 1];
        const long bi = in[b].c[0] >> in[b].l, bj = in[b].c[1] >> in[b].l, bk = in[b].c[2] >> in[b].lp;
        if (bi >= T.nb[0] || bj >= T.nb[1] || bk >= T.nb[2]) return set_error(HAMR_EINVAL, "block %d lies outside the domain", b);
        int* cc = &bcells[3 * ((bk * T.nb[1] + bj) * T.nb[0] + bi)];
        for (int d = 0; d < 3; d++) {
            if (cc[d] && cc[d] != nn[d])
                return set_error(HAMR_EINVAL, "block %d: cell counts differ from another block of its base block", b);
            cc[d] = nn[d];
        }
    }
    // requirements: each slot the target of the input block covering it; every slot covered once
    T.req.assign(units, (int8_t)-1);
    for (int b = 0; b < n; b++) {
        // one level of change per call: a regrid prolongs or restricts by a factor of 2
        const int8_t t = (int8_t)std::min(std::max(std::min(std::max(target[b], 0), T.Lf), in[b].l - 1), in[b].l + 1);
        long lo[3], hh[3];
        slot_box(T, in[b], lo, hh);
        for (long z = lo[2]; z < hh[2]; z++)
            for (long y = lo[1]; y < hh[1]; y++)
                for (long x = lo[0]; x < hh[0]; x++) {
                    if (x >= T.U[0] || y >= T.U[1] || z >= T.U[2])
                        return set_error(HAMR_EINVAL, "block %d lies outside the domain", b);
                    int8_t& r = T.req[T.idx(x, y, z)];
                    if (r >= 0) return set_error(HAMR_EINVAL, "block %d overlaps another block", b);
                    r = t;
                }
    }
    for (long u = 0; u < units; u++)
        if (T.req[u] < 0) return set_error(HAMR_EINVAL, "the blocks leave part of the domain uncovered");
    // nesting: face and edge neighbours more than a factor 2 apart in a direction refine the coarser one
    auto width = [&](const Blk& b, int d) {
        const long bi = b.c[0] >> b.l, bj = b.c[1] >> b.l, bk = b.c[2] >> b.lp;
        const int cells = bcells[3 * ((bk * T.nb[1] + bj) * T.nb[0] + bi) + d];
        return std::ldexp(base_ext[d], -((d == 2) ? b.lp : b.l)) / cells;
    };
    std::vector<Blk> leaves = all_leaves(T);
    bool stable = false;
    for (int it = 0; it < 64 && !stable; it++) {
        stable = true;
        std::vector<long> lo(3 * leaves.size()), hh(3 * leaves.size());
        for (size_t q = 0; q < leaves.size(); q++) slot_box(T, leaves[q], &lo[3 * q], &hh[3 * q]);
        for (size_t a = 0; a < leaves.size(); a++)
            for (size_t c = a + 1; c < leaves.size(); c++) {
                int ov = 0, to = 0;
                for (int d = 0; d < 3; d++) {
                    const int k = contact(lo[3 * a + d], hh[3 * a + d], lo[3 * c + d], hh[3 * c + d], T.U[d], T.per[d]);
                    if (k == 2) ov++;
                    else if (k == 1) to++;
                }
                if (ov + to < 3 || ov == 3 || to == 3) continue;  // apart, the same block, or a corner
                for (int d = 0; d < 3; d++) {
                    const double wa = width(leaves[a], d), wc = width(leaves[c], d);
                    if (wa > 2.0 * wc * (1.0 + 1e-9) && leaves[a].l < T.Lf) {
                        T.raise(leaves[a], leaves[a].l + 1);
                        stable = false;
                    } else if (wc > 2.0 * wa * (1.0 + 1e-9) && leaves[c].l < T.Lf) {
                        T.raise(leaves[c], leaves[c].l + 1);
                        stable = false;
                    }
                }
            }
        if (!stable) leaves = all_leaves(T);
    }
    if (!stable) return set_error(HAMR_EINVAL, "hamr_tree_adapt: the nesting rule did not settle");
    int lmax = 0;
    for (const Blk& f : leaves) lmax = std::max(lmax, f.l);
    *nout = (int)leaves.size();
    if (!out || (int)leaves.size() > cap)
        return set_error(HAMR_EINVAL, "output capacity %d, %zu blocks needed", cap, leaves.size());
    for (size_t q = 0; q < leaves.size(); q++) {
        const Blk& f = leaves[q];
        hamr_block_desc& B = out[q];
        const long bi = f.c[0] >> f.l, bj = f.c[1] >> f.l, bk = f.c[2] >> f.lp;
        const int* cc = &bcells[3 * ((bk * T.nb[1] + bj) * T.nb[0] + bi)];
        B.n1 = cc[0];
        B.n2 = cc[1];
        B.n3 = cc[2];
        double x0[3], h[3];
        for (int d = 0; d < 3; d++) {
            const int l = (d == 2) ? f.lp : f.l;
            const double ext = std::ldexp(base_ext[d], -l);
            x0[d] = dlo[d] + f.c[d] * ext;
            h[d] = ext / cc[d];
            const long nlev = (long)T.nb[d] << l;
            B.bc[2 * d] = (f.c[d] == 0) ? dbc[2 * d] : HAMR_BC_BLOCK;
            B.bc[2 * d + 1] = (f.c[d] == nlev - 1) ? dbc[2 * d + 1] : HAMR_BC_BLOCK;
        }
        B.x1min = x0[0];
        B.x2min = x0[1];
        B.x3min = x0[2];
        B.dx1 = h[0];
        B.dx2 = h[1];
        B.dx3 = h[2];
        B.lat = lmax - f.l;
    }
    return HAMR_OK;
}

}  // namespace

extern "C" int hamr_tree_adapt(const hamr_block_desc* cur, int n, const int* target, const double dlo[3],
                               const double base_ext[3], const int periodic[3], hamr_block_desc* out, int cap,
                               int* nout) {
    const int axis[2] = {0, 0};
    return adapt(cur, n, target, dlo, base_ext, periodic, axis, out, cap, nout);
}

extern "C" int hamr_tree_adapt_polar(const hamr_block_desc* cur, int n, const int* target, const double dlo[3],
                                     const double base_ext[3], const int periodic[3], const int axis[2],
                                     hamr_block_desc* out, int cap, int* nout) {
    if (!axis) return hamr::set_error(HAMR_EINVAL, "hamr_tree_adapt_polar: axis must not be NULL");
    return adapt(cur, n, target, dlo, base_ext, periodic, axis, out, cap, nout);
}
