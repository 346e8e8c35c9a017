// tree.cu -- host-side octree adaptation (Sec. 3.2): per-block target levels
// to a block tree that obeys the paper's nesting rule (a block's face and edge
// neighbours are at most one level coarser), ready for hamr_grid_regrid. A
// call moves each region by at most one level toward its target (the regrid
// prolongs and restricts by factors of 2); repeat until the tree is stable.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "hamr_internal.h"

namespace {

constexpr int MAX_LEVEL = 10;
constexpr long MAX_UNITS = 1L << 26;  // finest-level block slots of the domain

struct Tree {
    int nb[3];      // base blocks per direction
    int Lf;         // finest level
    long U[3];      // finest-level block slots per direction
    bool per[3];
    std::vector<int8_t> req;  // required level per finest slot
    long idx(long x, long y, long z) const { return (z * U[1] + y) * U[0] + x; }
    // largest requirement over the slots of a level-l block at coordinates c
    int max_req(int l, const long c[3]) const {
        const long s = 1L << (Lf - l);
        int m = 0;
        for (long z = c[2] * s; z < (c[2] + 1) * s; z++)
            for (long y = c[1] * s; y < (c[1] + 1) * s; y++)
                for (long x = c[0] * s; x < (c[0] + 1) * s; x++) m = std::max<int>(m, req[idx(x, y, z)]);
        return m;
    }
};

struct Leaf {
    int l;
    long c[3];
};

// leaves of a base block (coordinates cb at level 0): split while a slot needs more
void leaves_of(const Tree& T, int l, const long c[3], std::vector<Leaf>& out) {
    if (l < T.Lf && T.max_req(l, c) > l) {
        for (int kc = 0; kc < 2; kc++)
            for (int jc = 0; jc < 2; jc++)
                for (int ic = 0; ic < 2; ic++) {
                    const long cc[3] = {2 * c[0] + ic, 2 * c[1] + jc, 2 * c[2] + kc};
                    leaves_of(T, l + 1, cc, out);
                }
        return;
    }
    out.push_back(Leaf{l, {c[0], c[1], c[2]}});
}

std::vector<Leaf> all_leaves(const Tree& T) {
    std::vector<Leaf> out;
    for (long kb = 0; kb < T.nb[2]; kb++)
        for (long jb = 0; jb < T.nb[1]; jb++)
            for (long ib = 0; ib < T.nb[0]; ib++) {
                const long c[3] = {ib, jb, kb};
                leaves_of(T, 0, c, out);
            }
    return out;
}

// raises the requirement next to every leaf (faces and edges) to its level - 1; true if any changed
bool enforce_nesting(Tree& T, const std::vector<Leaf>& leaves) {
    bool changed = false;
    for (const Leaf& f : leaves) {
        if (f.l < 2) continue;
        const int need = f.l - 1;
        const long s = 1L << (T.Lf - f.l);
        for (int oz = -1; oz <= 1; oz++)
            for (int oy = -1; oy <= 1; oy++)
                for (int ox = -1; ox <= 1; ox++) {
                    const int nz = (ox != 0) + (oy != 0) + (oz != 0);
                    if (nz == 0 || nz == 3) continue;  // faces and edges, not corners
                    const int o[3] = {ox, oy, oz};
                    long lo[3];
                    bool inside = true;
                    for (int d = 0; d < 3; d++) {
                        lo[d] = (f.c[d] + o[d]) * s;
                        if (lo[d] < 0 || lo[d] >= T.U[d]) {
                            if (!T.per[d]) inside = false;
                            lo[d] = (lo[d] % T.U[d] + T.U[d]) % T.U[d];
                        }
                    }
                    if (!inside) continue;
                    for (long z = lo[2]; z < lo[2] + s; z++)
                        for (long y = lo[1]; y < lo[1] + s; y++)
                            for (long x = lo[0]; x < lo[0] + s; x++) {
                                int8_t& r = T.req[T.idx(x, y, z)];
                                if (r < need) {
                                    r = (int8_t)need;
                                    changed = true;
                                }
                            }
                }
    }
    return changed;
}

}  // namespace

extern "C" int hamr_tree_adapt(const hamr_block_desc* cur, int n, const int* target, const double dlo[3],
                               const double base_ext[3], const int periodic[3], hamr_block_desc* out, int cap,
                               int* nout) {
    using hamr::set_error;
    if (!cur || n < 1 || !target || !dlo || !base_ext || !periodic || !nout)
        return set_error(HAMR_EINVAL, "hamr_tree_adapt: NULL argument or n < 1");
    *nout = 0;
    const int cn[3] = {cur[0].n1, cur[0].n2, cur[0].n3};
    Tree T;
    T.Lf = 0;
    double hi[3] = {dlo[0], dlo[1], dlo[2]};
    std::vector<Leaf> in(n);
    int dbc[6] = {HAMR_BC_OUTFLOW, HAMR_BC_OUTFLOW, HAMR_BC_OUTFLOW, HAMR_BC_OUTFLOW, HAMR_BC_OUTFLOW,
                  HAMR_BC_OUTFLOW};
    for (int b = 0; b < n; b++) {
        const hamr_block_desc& B = cur[b];
        const int nn[3] = {B.n1, B.n2, B.n3};
        const double x0[3] = {B.x1min, B.x2min, B.x3min}, h[3] = {B.dx1, B.dx2, B.dx3};
        int L = -1;
        for (int d = 0; d < 3; d++) {
            if (nn[d] != cn[d]) return set_error(HAMR_EINVAL, "block %d: every block must have the same cell counts", b);
            const double ext = nn[d] * h[d];
            const int l = (int)std::lround(std::log2(base_ext[d] / ext));
            if (l < 0 || l > MAX_LEVEL || std::fabs(std::ldexp(ext, l) - base_ext[d]) > 1e-9 * base_ext[d])
                return set_error(HAMR_EINVAL, "block %d: extent is not base_ext / 2^L (L <= %d)", b, MAX_LEVEL);
            if (L >= 0 && l != L) return set_error(HAMR_EINVAL, "block %d: levels differ between directions", b);
            L = l;
            const double c = (x0[d] - dlo[d]) / ext;
            in[b].c[d] = std::lround(c);
            if (std::fabs(c - (double)in[b].c[d]) > 1e-6 || in[b].c[d] < 0)
                return set_error(HAMR_EINVAL, "block %d: not on the level-%d block lattice", b, l);
            hi[d] = std::max(hi[d], x0[d] + ext);
            if (std::fabs(x0[d] - dlo[d]) <= 1e-9 * base_ext[d]) dbc[2 * d] = B.bc[2 * d];
        }
        in[b].l = L;
        T.Lf = std::max(T.Lf, L);
        T.Lf = std::max(T.Lf, std::min(std::max(target[b], 0), MAX_LEVEL));
        if (target[b] > MAX_LEVEL) return set_error(HAMR_EINVAL, "block %d: target level above %d", b, MAX_LEVEL);
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
    // the upper domain faces' bc
    for (int b = 0; b < n; b++) {
        const hamr_block_desc& B = cur[b];
        const double x0[3] = {B.x1min, B.x2min, B.x3min}, h[3] = {B.dx1, B.dx2, B.dx3};
        for (int d = 0; d < 3; d++)
            if (std::fabs(x0[d] + cn[d] * h[d] - hi[d]) <= 1e-9 * base_ext[d]) dbc[2 * d + 1] = B.bc[2 * d + 1];
    }
    // requirements: each slot the target of the input block covering it; every slot covered once
    T.req.assign(units, (int8_t)-1);
    for (int b = 0; b < n; b++) {
        const long s = 1L << (T.Lf - in[b].l);
        // one level of change per call: a regrid prolongs or restricts by a factor of 2
        const int8_t t = (int8_t)std::min(std::max(std::min(std::max(target[b], 0), T.Lf), in[b].l - 1), in[b].l + 1);
        for (long z = in[b].c[2] * s; z < (in[b].c[2] + 1) * s; z++)
            for (long y = in[b].c[1] * s; y < (in[b].c[1] + 1) * s; y++)
                for (long x = in[b].c[0] * s; x < (in[b].c[0] + 1) * s; x++) {
                    if (x >= T.U[0] || y >= T.U[1] || z >= T.U[2])
                        return set_error(HAMR_EINVAL, "block %d lies outside the domain", b);
                    int8_t& r = T.req[T.idx(x, y, z)];
                    if (r >= 0) return set_error(HAMR_EINVAL, "block %d overlaps another block", b);
                    r = t;
                }
    }
    for (long u = 0; u < units; u++)
        if (T.req[u] < 0) return set_error(HAMR_EINVAL, "the blocks leave part of the domain uncovered");
    std::vector<Leaf> leaves = all_leaves(T);
    for (int it = 0; it < 64 && enforce_nesting(T, leaves); it++) leaves = all_leaves(T);
    int lmax = 0;
    for (const Leaf& f : leaves) lmax = std::max(lmax, f.l);
    *nout = (int)leaves.size();
    if (!out || (int)leaves.size() > cap)
        return set_error(HAMR_EINVAL, "output capacity %d, %zu blocks needed", cap, leaves.size());
    for (size_t q = 0; q < leaves.size(); q++) {
        const Leaf& f = leaves[q];
        hamr_block_desc& B = out[q];
        B.n1 = cn[0];
        B.n2 = cn[1];
        B.n3 = cn[2];
        double x0[3], h[3];
        for (int d = 0; d < 3; d++) {
            const double ext = std::ldexp(base_ext[d], -f.l);
            x0[d] = dlo[d] + f.c[d] * ext;
            h[d] = ext / cn[d];
            const long nlev = (long)T.nb[d] << f.l;
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
