"""Pins of the oracle's regridding (Sec. 3.2: prolongation and restriction on
(de)refinement; Balsara 2001 for the face field): a regrid onto the same tree
is the identity, refining then derefining returns the state, prolonged face
fields are divergence-free cell by cell and match the coarse faces, linear
fields are prolonged exactly, and restriction is the volume / area mean."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

NG = O.NG
PHYS = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_MINKOWSKI, gam=5.0 / 3.0, cour=0.5, floors=0)


def ora_blocks(blocks):
    return [O.make_block(b["n1"], b["n2"], b["n3"], b["x1min"], b["x2min"], b["x3min"], b["dx1"], b["dx2"],
                         b["dx3"], b["bc"], b["lat"]) for b in blocks]


def grid(blocks, states):
    a = O.AmrGrid(PHYS, ora_blocks(blocks))
    for i, (p, bf) in enumerate(states):
        a.set(i, p, bf)
    return a


def interior(b, p):
    return p[:, NG:NG + b["n3"], NG:NG + b["n2"], NG:NG + b["n1"]]


def faces(b, bf):
    n1, n2, n3 = b["n1"], b["n2"], b["n3"]
    return [bf[0][NG:NG + n3, NG:NG + n2, NG:NG + n1 + 1], bf[1][NG:NG + n3, NG:NG + n2 + 1, NG:NG + n1],
            bf[2][NG:NG + n3 + 1, NG:NG + n2, NG:NG + n1]]


def div_b(b, bf):
    f = faces(b, bf)
    return (np.diff(f[0], axis=2) / b["dx1"] + np.diff(f[1], axis=1) / b["dx2"] + np.diff(f[2], axis=0) / b["dx3"])


def test_regrid_onto_the_same_tree_is_the_identity():
    """Cells bitwise; faces bitwise except those a coarse block shares with finer ones, which take the
    mean of the finer faces (equal to the coarse face up to the rounding of the initial state)."""
    blocks = W.flat_box_tree(base=(2, 2, 2), n=6, refine=((0, 0, 0),))
    a = grid(blocks, W.flat_box_state(blocks))
    r = a.regrid(ora_blocks(blocks))
    for i, b in enumerate(blocks):
        p0, b0 = a.get(i)
        p1, b1 = r.get(i)
        assert np.array_equal(interior(b, p0)[:5], interior(b, p1)[:5]), i
        for x, y in zip(faces(b, b0), faces(b, b1)):
            if b["dx1"] < 0.06:  # the refined octant's children
                assert np.array_equal(x, y), i
            else:
                assert np.abs(x - y).max() <= 1e-14 * np.abs(b0).max(), i


@pytest.mark.parametrize("which", [(0, 0, 0), (1, 0, 1)])
def test_refine_then_derefine_returns_the_state(which):
    coarse = W.flat_box_tree(base=(2, 2, 2), n=6, refine=())
    fine = W.flat_box_tree(base=(2, 2, 2), n=6, refine=(which,))
    a = grid(coarse, W.flat_box_state(coarse))
    back = a.regrid(ora_blocks(fine)).regrid(ora_blocks(coarse))
    for i, b in enumerate(coarse):
        p0, b0 = a.get(i)
        p1, b1 = back.get(i)
        x, y = interior(b, p0)[:5], interior(b, p1)[:5]
        assert np.abs(x - y).max() <= 1e-14 * np.abs(x).max(), i
        for f0, f1 in zip(faces(b, b0), faces(b, b1)):
            assert np.abs(f0 - f1).max() <= 1e-14 * np.abs(b0).max(), i


def test_prolonged_field_is_divergence_free_and_matches_the_coarse_faces():
    coarse = W.flat_box_tree(base=(2, 2, 2), n=6, refine=())
    fine = W.flat_box_tree(base=(2, 2, 2), n=6, refine=((1, 1, 0),))
    a = grid(coarse, W.flat_box_state(coarse, bamp=0.2))
    r = a.regrid(ora_blocks(fine))
    bmax = max(np.abs(a.get(i)[1]).max() for i in range(len(coarse)))
    for i, b in enumerate(fine):
        _, bf = r.get(i)
        assert np.abs(div_b(b, bf)).max() <= 1e-12 * bmax / b["dx1"], i
    # a coarse x1-face on the refined block's lower x boundary is the mean of the 4 fine faces on it
    ci = next(i for i, b in enumerate(coarse) if (b["x1min"], b["x2min"], b["x3min"]) == (0.5, 0.5, 0.0))
    _, cb = a.get(ci)
    cf = faces(coarse[ci], cb)[0][:, :, 0]
    fine_lo = [i for i, b in enumerate(fine) if b["x1min"] == 0.5 and b["dx1"] < coarse[0]["dx1"]]
    acc = np.zeros_like(cf)
    for i in fine_lo:
        b = fine[i]
        ff = faces(b, r.get(i)[1])[0][:, :, 0]  # (n3, n2) fine faces at x = 0.5
        j0 = int(round((b["x2min"] - 0.5) / (2 * b["dx2"])))
        k0 = int(round(b["x3min"] / (2 * b["dx3"])))
        m3, m2 = ff.shape
        acc[k0:k0 + m3 // 2, j0:j0 + m2 // 2] += 0.25 * (ff[0::2, 0::2] + ff[1::2, 0::2] + ff[0::2, 1::2] +
                                                          ff[1::2, 1::2])
    assert np.abs(acc - cf).max() <= 1e-14 * bmax


def test_refinement_next_to_existing_fine_blocks_stays_divergence_free():
    """Refining a block whose neighbour is already fine: the new fine faces on the shared plane are the
    neighbour's faces (copied), and the interior fine faces are corrected so that every fine cell is
    divergence-free (the coarse face's linear profile alone would leave each fine cell with a
    divergence of the size of the neighbour's sub-face variation)."""
    old = W.flat_box_tree(base=(2, 2, 2), n=6, refine=((0, 0, 0),))
    new = W.flat_box_tree(base=(2, 2, 2), n=6, refine=((0, 0, 0), (1, 0, 0)))
    a = grid(old, W.flat_box_state(old, bamp=0.3))
    a.period()  # the fine and coarse faces at the shared plane have been synchronised by a step
    r = a.regrid(ora_blocks(new))
    bmax = max(np.abs(r.get(i)[1]).max() for i in range(len(new)))
    for i, b in enumerate(new):
        _, bf = r.get(i)
        assert np.abs(div_b(b, bf)).max() <= 1e-12 * bmax / b["dx1"], i
    # faces on x = 0.5 of the new fine blocks equal the old fine faces there
    fine_old = {(b["x2min"], b["x3min"]): i for i, b in enumerate(old) if b["dx1"] < 0.06 and b["x1min"] > 0.2}
    for i, b in enumerate(new):
        if b["dx1"] < 0.06 and b["x1min"] == 0.5:
            j = fine_old[(b["x2min"], b["x3min"])]
            got = faces(b, r.get(i)[1])[0][:, :, 0]
            want = faces(old[j], a.get(j)[1])[0][:, :, -1]
            assert np.array_equal(got, want), i


def _linear_states(blocks, c=(0.1, -0.05, 0.02), g=0.3):
    """rho, u linear in x; face field B = (1 + g x, 0.5 - g y, 0.2) (divergence-free, linear)."""
    out = []
    for b in blocks:
        shp = (b["n3"] + 2 * NG, b["n2"] + 2 * NG, b["n1"] + 2 * NG)
        p = np.zeros((8,) + shp)
        bf = np.zeros((3,) + shp)
        x = b["x1min"] + (np.arange(-NG, b["n1"] + NG) + 0.5) * b["dx1"]
        y = b["x2min"] + (np.arange(-NG, b["n2"] + NG) + 0.5) * b["dx2"]
        z = b["x3min"] + (np.arange(-NG, b["n3"] + NG) + 0.5) * b["dx3"]
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        p[0] = 1.0 + c[0] * X + c[1] * Y + c[2] * Z
        p[1] = 2.0 + c[1] * X - c[2] * Z
        p[2] = 0.1 * X
        xf = b["x1min"] + np.arange(-NG, b["n1"] + NG) * b["dx1"]
        yf = b["x2min"] + np.arange(-NG, b["n2"] + NG) * b["dx2"]
        Zc, Yc, Xf = np.meshgrid(z, y, xf, indexing="ij")
        bf[0] = 1.0 + g * Xf
        Zc, Yf, Xc = np.meshgrid(z, yf, x, indexing="ij")
        bf[1] = 0.5 - g * Yf
        bf[2] = 0.2
        out.append((p, bf))
    return out


def test_linear_fields_are_prolonged_exactly():
    """Away from the old block's edges (where a slope stencil would leave the block and the slope is 0),
    MINMOD prolongation of linear cell data and the Balsara prolongation of a linear divergence-free
    face field reproduce them exactly."""
    coarse = W.flat_box_tree(base=(2, 2, 2), n=8, refine=())
    fine = W.flat_box_tree(base=(2, 2, 2), n=8, refine=((0, 0, 0),))
    a = grid(coarse, _linear_states(coarse))
    r = a.regrid(ora_blocks(fine))
    want = _linear_states(fine)
    for i, b in enumerate(fine):
        if b["dx1"] > 0.05:
            continue
        p, bf = r.get(i)
        pw, bw = want[i]
        # fine cells 2..n-3 of each child lie in coarse cells with both neighbours inside the old block
        sl = (slice(None), slice(NG + 2, NG + b["n3"] - 2), slice(NG + 2, NG + b["n2"] - 2),
              slice(NG + 2, NG + b["n1"] - 2))
        x0 = b["x1min"] == 0.0
        s1 = slice(NG + 2, NG + b["n1"] - 2)
        assert np.abs(p[:3][sl[0:1] + sl[1:]] - pw[:3][sl[0:1] + sl[1:]]).max() < 1e-14, (i, x0, s1)
        for d in range(3):
            fs = [slice(NG + 2, NG + b["n3"] - 2), slice(NG + 2, NG + b["n2"] - 2), slice(NG + 2, NG + b["n1"] - 2)]
            assert np.abs(bf[d][tuple(fs)] - bw[d][tuple(fs)]).max() < 1e-14, (i, d)


def test_restriction_is_the_mean():
    fine = W.flat_box_tree(base=(2, 2, 2), n=4, refine=((1, 1, 1),))
    coarse = W.flat_box_tree(base=(2, 2, 2), n=4, refine=())
    states = W.flat_box_state(fine, amp=0.2)
    a = grid(fine, states)
    r = a.regrid(ora_blocks(coarse))
    ci = next(i for i, b in enumerate(coarse) if (b["x1min"], b["x2min"], b["x3min"]) == (0.5, 0.5, 0.5))
    pc, bc = r.get(ci)
    kids = [i for i, b in enumerate(fine) if b["dx1"] < 0.1]
    b0 = fine[kids[0]]
    for i in kids:
        b = fine[i]
        p, bf = a.get(i)
        ic = int(round((b["x1min"] - 0.5) / b["dx1"] / 2))
        jc = int(round((b["x2min"] - 0.5) / b["dx2"] / 2))
        kc = int(round((b["x3min"] - 0.5) / b["dx3"] / 2))
        q = interior(b, p)[:5]
        mean = 0.125 * sum(q[:, a3::2, a2::2, a1::2] for a1 in (0, 1) for a2 in (0, 1) for a3 in (0, 1))
        m2, m3 = b["n1"] // 2, b["n3"] // 2
        got = interior(coarse[ci], pc)[:5][:, kc:kc + m3, jc:jc + m3, ic:ic + m2]
        assert np.abs(got - mean).max() <= 1e-14 * np.abs(mean).max(), i
        f1 = faces(b, bf)[0]
        fm = 0.25 * (f1[0::2, 0::2, 0::2] + f1[1::2, 0::2, 0::2] + f1[0::2, 1::2, 0::2] + f1[1::2, 1::2, 0::2])
        gf = faces(coarse[ci], bc)[0][kc:kc + m3, jc:jc + m3, ic:ic + m2 + 1]
        assert np.abs(gf - fm).max() <= 1e-14 * np.abs(fm).max() + 1e-300, i
    del b0


# ---- 6-way splits (Sec. 3.3.1): two children keep the parent's x3 cells, four halve all three widths;
# in a periodic flat box with the 'axis' on the split block's lower x2 side (workloads.split6)

def test_six_way_split_then_merge_returns_the_state():
    coarse = W.flat_box_tree(base=(2, 2, 2), n=6, refine=())
    split = W.flat_box_tree6(base=(2, 2, 2), n=6, split=((1, 0, 1),))
    assert len(split) == 13
    a = grid(coarse, W.flat_box_state(coarse, bamp=0.2))
    back = a.regrid(ora_blocks(split)).regrid(ora_blocks(coarse))
    for i, b in enumerate(coarse):
        p0, b0 = a.get(i)
        p1, b1 = back.get(i)
        x, y = interior(b, p0)[:5], interior(b, p1)[:5]
        assert np.abs(x - y).max() <= 1e-14 * np.abs(x).max(), i
        for f0, f1 in zip(faces(b, b0), faces(b, b1)):
            assert np.abs(f0 - f1).max() <= 1e-14 * np.abs(b0).max(), i


def test_six_way_children_are_divergence_free_and_match_the_coarse_faces():
    coarse = W.flat_box_tree(base=(2, 2, 2), n=6, refine=())
    split = W.flat_box_tree6(base=(2, 2, 2), n=6, split=((0, 1, 0),))
    a = grid(coarse, W.flat_box_state(coarse, bamp=0.2))
    r = a.regrid(ora_blocks(split))
    bmax = max(np.abs(a.get(i)[1]).max() for i in range(len(coarse)))
    kinds = set()
    for i, b in enumerate(split):
        _, bf = r.get(i)
        assert np.abs(div_b(b, bf)).max() <= 1e-12 * bmax / b["dx1"], i
        kinds.add((round(b["dx1"], 9), round(b["dx3"], 9)))
    assert len(kinds) == 3   # base blocks, children keeping x3, children halving x3
    # the coarse x2-face at y = 0.5 (the split block's lower, 'axis' side) is the mean of the axis children's
    # faces on it: 2 x 1 fine faces (x1 halves, the whole x3 cell) per coarse face
    ci = next(i for i, b in enumerate(coarse) if (b["x1min"], b["x2min"], b["x3min"]) == (0.0, 0.5, 0.0))
    cf = faces(coarse[ci], a.get(ci)[1])[1][:, 0, :]          # (n3, n1)
    acc = np.zeros_like(cf)
    for i, b in enumerate(split):
        if b["x2min"] == 0.5 and b["dx1"] < coarse[0]["dx1"] and b["dx3"] == coarse[0]["dx3"]:
            ff = faces(b, r.get(i)[1])[1][:, 0, :]               # (n3, n1) fine faces at y = 0.5
            i0 = int(round(b["x1min"] / (2 * b["dx1"])))
            m1 = ff.shape[1] // 2
            acc[:, i0:i0 + m1] += 0.5 * (ff[:, 0::2] + ff[:, 1::2])
    assert np.abs(acc - cf).max() <= 1e-14 * bmax


def test_six_way_split_next_to_fine_blocks_stays_divergence_free():
    """The interior-face correction on 2 x 2 x 1 fine cells (the axis children) and 2 x 2 x 2 (the
    others), with an octree-refined neighbour across x1 whose faces are kept on the shared plane."""
    old = W.flat_box_tree6(base=(2, 2, 2), n=6, refine=((0, 0, 0),), split=())
    new = W.flat_box_tree6(base=(2, 2, 2), n=6, refine=((0, 0, 0),), split=((1, 0, 0),))
    a = grid(old, W.flat_box_state(old, bamp=0.3))
    a.period()
    r = a.regrid(ora_blocks(new))
    bmax = max(np.abs(r.get(i)[1]).max() for i in range(len(new)))
    for i, b in enumerate(new):
        _, bf = r.get(i)
        assert np.abs(div_b(b, bf)).max() <= 1e-12 * bmax / b["dx1"], i


def test_six_way_children_prolong_linear_fields_exactly():
    coarse = W.flat_box_tree(base=(2, 2, 2), n=8, refine=())
    split = W.flat_box_tree6(base=(2, 2, 2), n=8, split=((0, 0, 0),))
    a = grid(coarse, _linear_states(coarse))
    r = a.regrid(ora_blocks(split))
    want = _linear_states(split)
    for i, b in enumerate(split):
        if b["dx1"] > 0.05:
            continue
        p, bf = r.get(i)
        pw, bw = want[i]
        sl = (slice(0, 3), slice(NG + 2, NG + b["n3"] - 2), slice(NG + 2, NG + b["n2"] - 2),
              slice(NG + 2, NG + b["n1"] - 2))
        assert np.abs(p[sl] - pw[sl]).max() < 1e-14, i
        for d in range(3):
            fs = (slice(NG + 2, NG + b["n3"] - 2), slice(NG + 2, NG + b["n2"] - 2), slice(NG + 2, NG + b["n1"] - 2))
            assert np.abs(bf[d][fs] - bw[d][fs]).max() < 1e-14, (i, d)


@pytest.mark.parametrize("src,dst", [(dict(split=((0, 0, 0),)), dict(refine=((0, 0, 0),), split=())),
                                     (dict(refine=((0, 0, 0),), split=()), dict(split=((0, 0, 0),))),
                                     (dict(split=((0, 1, 0),)), dict(split=((0, 0, 0),))),
                                     (dict(split=((0, 0, 0), (1, 1, 0))), dict(split=((1, 0, 0), (0, 1, 1))))])
def test_x3_only_refinement_and_merge_stay_divergence_free(src, dst):
    """A region whose cells change along x3 alone (the axis children of a 6-way split becoming octants,
    and back), and splits next to merges: the refinement takes Balsara's polynomial on 1 x 1 x 2 fine
    cells, the merge the area means; every cell stays divergence-free. Two versions failed these:
    piecewise-constant copies of the x1 and x2 faces along x3 (the x3 faces change across the cell),
    and octants whose faces on a plane shared with an axis child were copied piecewise-constant along
    x3 while the axis child's side of the plane took its polynomial's linear profile."""
    old = W.flat_box_tree6(base=(2, 2, 2), n=6, **src)
    new = W.flat_box_tree6(base=(2, 2, 2), n=6, **dst)
    a = grid(old, W.flat_box_state(old, bamp=0.2))
    a.period()
    r = a.regrid(ora_blocks(new))
    bmax = max(np.abs(r.get(i)[1]).max() for i in range(len(new)))
    for i, b in enumerate(new):
        _, bf = r.get(i)
        assert np.abs(div_b(b, bf)).max() <= 1e-12 * bmax / b["dx1"], i
