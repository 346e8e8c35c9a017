"""Pins of the oracle's internal SMR inside the multi-block step (Sec. 3.3.2 with
Sec. 3.2 and 3.4): a torus split into same-level blocks steps like the single
block with the same grouping; across a refined polar block (6-way split) and
local time steps the groups of the two resolutions cover the same phi ranges,
so every face shared by two blocks keeps one value (the coarse face equals the
mean of the finer faces covering it), grouped cells stay identical, mass is
conserved to round-off and div B stays at round-off."""
import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

from helpers import NG, ora_tree, polar_field, refined_polar_tree, torus_case

GAM = 5.0 / 3.0


def _split(prim, bf, d, nb=(2, 2, 2)):
    """the single-block torus cut into nb same-level blocks: oracle blocks and their padded states"""
    N = (d.n1, d.n2, d.n3)
    n = [N[e] // nb[e] for e in range(3)]
    blocks, states = [], []
    for kb in range(nb[2]):
        for jb in range(nb[1]):
            for ib in range(nb[0]):
                bc = [4] * 6
                if ib == 0:
                    bc[0] = O.BC_OUTFLOW_NOINFLOW
                if ib == nb[0] - 1:
                    bc[1] = O.BC_OUTFLOW_NOINFLOW
                if jb == 0:
                    bc[2] = O.BC_POLAR
                if jb == nb[1] - 1:
                    bc[3] = O.BC_POLAR
                if kb == 0:
                    bc[4] = O.BC_PERIODIC
                if kb == nb[2] - 1:
                    bc[5] = O.BC_PERIODIC
                i0, j0, k0 = ib * n[0], jb * n[1], kb * n[2]
                blocks.append(O.make_block(n[0], n[1], n[2], d.x1min + i0 * d.dx1, d.x2min + j0 * d.dx2,
                                           d.x3min + k0 * d.dx3, d.dx1, d.dx2, d.dx3, bc, 0))
                pb = np.zeros((8, n[2] + 6, n[1] + 6, n[0] + 6))
                bb = np.zeros((3, n[2] + 6, n[1] + 6, n[0] + 6))
                pb[:, 3:3 + n[2], 3:3 + n[1], 3:3 + n[0]] = prim[:, 3 + k0:3 + k0 + n[2], 3 + j0:3 + j0 + n[1],
                                                                  3 + i0:3 + i0 + n[0]]
                bb[:, 3:4 + n[2], 3:4 + n[1], 3:4 + n[0]] = bf[:, 3 + k0:4 + k0 + n[2], 3 + j0:4 + j0 + n[1],
                                                                3 + i0:4 + i0 + n[0]]
                states.append(((i0, j0, k0), pb, bb))
    return blocks, states, n


@pytest.mark.parametrize("nb", [(2, 2, 2), (2, 4, 1)])
def test_torus_split_with_smr_matches_the_single_block(nb):
    """Eight (or eight theta-stacked) same-level blocks with two SMR levels: the block-tree path groups
    the same rows and phi ranges as the single block (a group mean, group inversion or CFL width
    missing from the tree path, or taken per block at the wrong rows, breaks this)."""
    geo, d, prim, bf = torus_case(32, 32, 16, seed=3)
    d.smr = 2
    polar_field(bf, d.x1min, d.x2min, d.x3min, d.dx1, d.dx2, d.dx3, (d.n1, d.n2, d.n3))
    blocks, states, n = _split(prim, bf, d, nb)
    a = O.AmrGrid(d, blocks)
    for b, (_, pb, bb) in enumerate(states):
        a.set(b, pb, bb)
    g = O.Grid(d)
    g.set(prim, bf)
    for _ in range(2):
        assert abs(g.step() - a.period()) == 0.0
    p1, b1 = g.get()
    num, den = np.zeros(8), np.zeros(8)
    fnum, fden = np.zeros(3), np.zeros(3)
    for b, ((i0, j0, k0), _, _) in enumerate(states):
        pb, bb = a.get(b)
        x = pb[:, 3:3 + n[2], 3:3 + n[1], 3:3 + n[0]]
        y = p1[:, 3 + k0:3 + k0 + n[2], 3 + j0:3 + j0 + n[1], 3 + i0:3 + i0 + n[0]]
        num += np.abs(x - y).reshape(8, -1).sum(1)
        den += np.abs(y).reshape(8, -1).sum(1)
        for m in range(3):
            e = [n[2], n[1], n[0]]
            e[2 - m] += 1
            xf = bb[m, 3:3 + e[0], 3:3 + e[1], 3:3 + e[2]]
            yf = b1[m, 3 + k0:3 + k0 + e[0], 3 + j0:3 + j0 + e[1], 3 + i0:3 + i0 + e[2]]
            fnum[m] += np.abs(xf - yf).sum()
            fden[m] += np.abs(yf).sum()
    assert num.sum() / den.sum() < 1e-13 and (num / den).max() < 1e-11, num / den
    assert (fnum / fden).max() < 1e-12, fnum / fden


def smr_width(b, j, smr, h2b, h3b):
    """group width of row j of block b (dict) under smr levels: the rows and phi ranges of the
    coarsest polar blocks (x2 width h2b, x3 width h3b), restated from the paper's level rule"""
    l2 = int(round(np.log2(h2b / b["dx2"])))
    l3 = int(round(np.log2(h3b / b["dx3"])))
    jp = 1 << 30
    if b["bc"][2] == O.BC_POLAR:
        jp = j
    if b["bc"][3] == O.BC_POLAR:
        jp = min(jp, b["n2"] - 1 - j)
    for lev in range(smr, 0, -1):
        if (jp >> l2) < 2 ** (smr - lev):
            return 2 ** lev * 2 ** l3
    return 1


def _refined_polar_case(smr):
    blocks, states = refined_polar_tree()
    phys = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_SPHERICAL, gam=GAM, cour=0.8, floors=0, smr=smr)
    return blocks, phys, ora_tree(phys, blocks, states)


def _mass_and_div(a, blocks, phys):
    mass, divmax = 0.0, 0.0
    for i, b in enumerate(blocks):
        p, bf = a.get(i)
        n1, n2, n3 = b["n1"], b["n2"], b["n3"]
        s = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
        x1 = b["x1min"] + (np.arange(n1) + 0.5) * b["dx1"]
        x2 = b["x2min"] + (np.arange(n2) + 0.5) * b["dx2"]
        pr = p[:, NG:NG + n3, NG:NG + n2, NG:NG + n1].reshape(8, -1).T
        U = O.p2u_many(phys, pr, np.broadcast_to(x1, (n3, n2, n1)).ravel(),
                       np.broadcast_to(x2[:, None], (n3, n2, n1)).ravel())
        mass += U[:, 0].sum() * b["dx1"] * b["dx2"] * b["dx3"]
        div = ((bf[0][NG:NG + n3, NG:NG + n2, NG + 1:NG + n1 + 1] - bf[0][s]) / b["dx1"]
               + (bf[1][NG:NG + n3, NG + 1:NG + n2 + 1, NG:NG + n1] - bf[1][s]) / b["dx2"]
               + (bf[2][NG + 1:NG + n3 + 1, NG:NG + n2, NG:NG + n1] - bf[2][s]) / b["dx3"])
        divmax = max(divmax, np.abs(div).max() / (np.abs(bf).max() / min(b["dx1"], b["dx2"], b["dx3"])))
    return mass, divmax


def _shared_x1_faces(a, blocks):
    """largest difference between a block's upper x1-faces and the finer or equal side's faces over
    the same area (mean over the coarser cell's extent), relative to the largest face value"""
    faces = [a.get(i)[1] for i in range(len(blocks))]
    worst, scale = 0.0, max(np.abs(f[0]).max() for f in faces)
    for i, p in enumerate(blocks):
        hi1 = p["x1min"] + p["n1"] * p["dx1"]
        for j, c in enumerate(blocks):
            if abs(c["x1min"] - hi1) > 1e-9:
                continue
            t0, t1 = max(p["x2min"], c["x2min"]), min(p["x2min"] + p["n2"] * p["dx2"], c["x2min"] + c["n2"] * c["dx2"])
            z0, z1 = max(p["x3min"], c["x3min"]), min(p["x3min"] + p["n3"] * p["dx3"], c["x3min"] + c["n3"] * c["dx3"])
            if t1 - t0 < 1e-9 or z1 - z0 < 1e-9:
                continue
            h2, h3 = max(p["dx2"], c["dx2"]), max(p["dx3"], c["dx3"])

            def mean_face(b, bf, i1, y, z):
                j0, j1 = (int(round((v - b["x2min"]) / b["dx2"])) for v in (y, y + h2))
                k0, k1 = (int(round((v - b["x3min"]) / b["dx3"])) for v in (z, z + h3))
                return bf[0][NG + k0:NG + k1, NG + j0:NG + j1, NG + i1].mean()

            for y in np.arange(t0, t1 - 1e-12, h2):
                for z in np.arange(z0, z1 - 1e-12, h3):
                    worst = max(worst, abs(mean_face(p, faces[i], p["n1"], y, z) - mean_face(c, faces[j], 0, y, z)))
    return worst / scale


def test_groups_coincide_across_a_refined_polar_block():
    """A polar block split 6-way next to coarser polar blocks, on a lower LAT level: after each period
    every shared x1-face has one value (the finer blocks group their rows by the coarse rows, so the
    EMFs the two sides exchange are averaged over the same phi ranges), every group's cells hold
    identical primitives, mass is conserved and div B stays at round-off."""
    smr = 1
    blocks, phys, a = _refined_polar_case(smr)
    assert len({b["lat"] for b in blocks}) > 1
    polar = [b for b in blocks if O.BC_POLAR in (b["bc"][2], b["bc"][3])]
    assert len({b["dx2"] for b in polar}) == 2  # two resolutions meet at the axis
    h2b, h3b = max(b["dx2"] for b in polar), max(b["dx3"] for b in polar)
    m0, d0 = _mass_and_div(a, blocks, phys)
    assert _shared_x1_faces(a, blocks) < 1e-14
    ngroups = 0
    for _ in range(3):
        a.period()
        m1, d1 = _mass_and_div(a, blocks, phys)
        assert abs(m1 - m0) <= 1e-13 * abs(m0) and d1 <= 1e-12
        assert _shared_x1_faces(a, blocks) <= 1e-13
        for i, b in enumerate(blocks):
            p, _ = a.get(i)
            for j in range(b["n2"]):
                w = smr_width(b, j, smr, h2b, h3b)
                if w == 1:
                    continue
                row = p[:5, NG:NG + b["n3"], NG + j, NG:NG + b["n1"]].reshape(5, b["n3"] // w, w, b["n1"])
                assert np.array_equal(row, np.broadcast_to(row[:, :, :1, :], row.shape)), (i, j, w)
                ngroups += b["n3"] // w * b["n1"]
    assert ngroups > 0
