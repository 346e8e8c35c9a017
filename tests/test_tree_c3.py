"""The C3 block tree (paper_1912_10192_gb300/workloads.py c3_tree) on the CPU:
512 blocks, the stated groups and cell counts, a 1024 x 512 x 512 effective
finest grid, blocks tiling the domain without overlap, and the nesting rule
of Sec. 3.2 (face and edge neighbours at most a factor 2 apart per
direction). The plan's literal shapes for the polar blocks (unrefined polar
base blocks of 32 x 16 x 8 cells, off-axis 6-way children of 32^3) break that
rule in phi and theta; the test records where, which is why the tree keeps
the polar rows at 32 x 32 x 16."""
import math
from collections import Counter

from paper_1912_10192_gb300 import workloads as W


def test_c3_tree_groups_cells_and_levels():
    blocks = W.c3_tree(n=32)
    s = W.tree_summary(blocks)
    assert s["blocks"] == 512 and s["cells"] == 13_107_200
    assert s["groups"] == {"base 32x32x32": 48, "level 1 32x32x32": 112, "level 2 32x32x32": 128,
                           "polar base 32x32x16": 32, "polar child on the axis 32x32x16": 64,
                           "polar child off the axis 32x32x16": 128}
    assert s["refinement_levels"] == {"0": 80, "1": 304, "2": 128}
    assert set(s["lat_levels"]) == {"0", "1", "2", "3"}
    # effective finest grid: the level-2 cell widths
    fine = [b for b in blocks if b["level"] == 2][0]
    ext = (math.log(50.0) - math.log(1.2), math.pi, 2 * math.pi)
    assert [round(ext[d] / fine["dx%d" % (d + 1)]) for d in range(3)] == [1024, 512, 512]


def test_c3_tree_tiles_the_domain_and_nests():
    blocks = W.c3_tree(n=32)
    ext = (math.log(50.0) - math.log(1.2), math.pi, 2 * math.pi)
    vol = sum(b["n1"] * b["dx1"] * b["n2"] * b["dx2"] * b["n3"] * b["dx3"] for b in blocks)
    assert abs(vol - ext[0] * ext[1] * ext[2]) <= 1e-9 * vol
    # no two blocks overlap: sample every block's cell centres on a coarse lattice of the finest grid
    owner = {}
    for i, b in enumerate(blocks):
        for a in range(2):
            for c in range(2):
                for e in range(2):
                    x = (b["x1min"] + (0.25 + 0.5 * a) * b["n1"] * b["dx1"],
                         b["x2min"] + (0.25 + 0.5 * c) * b["n2"] * b["dx2"],
                         b["x3min"] + (0.25 + 0.5 * e) * b["n3"] * b["dx3"])
                    key = tuple(int(x[d] / ext[d] * 4096) for d in range(3))
                    assert key not in owner, (i, owner.get(key))
                    owner[key] = i
    assert W.nesting_violations(blocks) == []
    # every block's LAT level differs by at most one from the blocks it touches
    for i, b in enumerate(blocks):
        for j, c in enumerate(blocks):
            if i < j and W._touch(b, c, 2 * math.pi):
                assert abs(b["lat"] - c["lat"]) <= 1


def test_literal_polar_shapes_break_the_nesting_rule():
    lit = W.c3_blocks(polar_cells=(32, 16, 8), far_cells=(32, 32, 32), axis_cells=(32, 32, 16))
    s = W.tree_summary(lit)
    assert s["blocks"] == 512 and s["cells"] == 14_811_136
    bad = Counter((lit[a]["group"], lit[c]["group"], d) for a, c, d, r in W.nesting_violations(lit))
    assert bad[("polar base", "base", 3)] > 0            # phi cells 4x wider than the equatorial base's
    assert bad[("polar child on the axis", "polar child off the axis", 3)] > 0
    assert any(k[0] == "polar base" and k[1].startswith("polar child") and k[2] == 2 for k in bad)


def test_c3_tree_with_internal_smr_widths_and_levels():
    """Internal SMR (Sec. 3.3.2) in the C3 polar rows: the first row of the coarsest polar blocks
    is grouped 4 wide with two levels, the second 2 wide, the rest not; the on-axis children (x2
    cells twice finer, x3 as coarse) group their first two rows 4 wide and the next two 2 wide;
    blocks off the axis group nothing. Wider cells in phi lift the light-crossing step of the polar
    rows (by about 3x with two levels, the r and theta terms left), and the tree keeps its LAT levels."""
    blocks = W.c3_tree(n=32)
    ws = W.smr_row_widths(blocks, 2)
    for b, w in zip(blocks, ws):
        if b["group"] == "polar base":
            first = list(w[:3]) if b["bc"][2] == 2 else list(w[::-1][:3])
            assert first == [4, 2, 1] and (w == 1).sum() == 30
        elif b["group"] == "polar child on the axis":
            first = list(w[:5]) if b["bc"][2] == 2 else list(w[::-1][:5])
            assert first == [4, 4, 2, 2, 1] and (w == 1).sum() == 28
        else:
            assert (w == 1).all(), b["group"]
    assert all((w == 1).all() for w in W.smr_row_widths(blocks, 0))
    lat0 = [b["lat"] for b in blocks]
    for smr in (1, 2, 3):
        assert [b["lat"] for b in W.c3_tree(n=32, smr=smr)] == lat0

    def fine_dt(smr):
        bl = W.c3_tree(n=32, smr=smr)
        out = []
        for b, w in zip(bl, W.smr_row_widths(bl, smr)):
            r = [math.exp(b["x1min"] + (i + 0.5) * b["dx1"]) for i in range(b["n1"])]
            th = [b["x2min"] + (j + 0.5) * b["dx2"] for j in range(b["n2"])]
            inv = max(1 / (ri * b["dx1"]) + 1 / (ri * b["dx2"]) + 1 / (ri * abs(math.sin(t)) * b["dx3"] * wj)
                      for ri in r for t, wj in zip(th, w))
            out.append(1 / inv / 2 ** b["lat"])
        return min(out)
    gain = fine_dt(2) / fine_dt(0)
    assert 2.5 < gain < 4.0, gain
