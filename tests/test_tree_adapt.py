"""The host-side octree adaptation (hamr_tree_adapt; Sec. 3.2: blocks meeting
the refinement criterion go to the highest level, their face and edge
neighbours to at most one level below, recursively): checked on CPU by the
properties that define it: the blocks tile the domain without overlap, every
region reaches its target, no face or edge neighbours differ by more than one
level, regions with no target and no nesting constraint stay at the base
level, and a tree whose targets drop is derefined. No GPU is needed."""
import itertools

import numpy as np
import pytest

from paper_1912_10192_gb300 import _build, hamr
from paper_1912_10192_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def _blocks(tree):
    return [hamr.block_from_dict(b) for b in tree]


def _box(b):
    lo = np.array([b.x1min, b.x2min, b.x3min])
    ext = np.array([b.n1 * b.dx1, b.n2 * b.dx2, b.n3 * b.dx3])
    return lo, lo + ext


def _level(b, base=0.25):
    return int(round(np.log2(base / (b.n1 * b.dx1))))


def _check_tree(out, volume=1.0, L=1.0):
    """Tiling (total volume, no overlap) and the one-level jump across faces and edges (periodic box)."""
    lo = np.array([_box(b)[0] for b in out])
    hi = np.array([_box(b)[1] for b in out])
    lev = np.array([_level(b) for b in out])
    assert abs(float(np.prod(hi - lo, axis=1).sum()) - volume) < 1e-12
    n = len(out)
    kind = np.zeros((n, n), dtype=int)  # 0 none, 1 face, 2 edge, 3 corner (smallest contact over shifts)
    for s in itertools.product((-L, 0.0, L), repeat=3):
        s = np.array(s)
        ext = np.minimum(hi[:, None, :], hi[None, :, :] + s) - np.maximum(lo[:, None, :], lo[None, :, :] + s)
        touch = np.all(ext > -1e-12, axis=2)
        flat = np.sum(np.abs(ext) <= 1e-12, axis=2)
        over = touch & (flat == 0)
        np.fill_diagonal(over, False) if not np.any(s) else None
        assert not np.any(over), "overlap"
        k = np.where(touch, flat, 0)
        kind = np.where((kind == 0) | ((k > 0) & (k < kind)), np.where(k > 0, k, kind), kind)
    np.fill_diagonal(kind, 0)
    jump = np.abs(lev[:, None] - lev[None, :])
    bad = ((kind == 1) | (kind == 2)) & (jump > 1)
    assert not np.any(bad), np.argwhere(bad)[:3]


def _adapt_until_stable(cur, target_of, calls=6):
    """Repeated adaptation (one level per call) with targets from block positions; the per-call level
    change is checked on the way."""
    for _ in range(calls):
        out = hamr.tree_adapt(cur, [target_of(b) for b in cur], (0, 0, 0), (0.25, 0.25, 0.25))
        for b in out:  # every new block moved at most one level from the blocks it overlaps
            lo, hi = _box(b)
            for c in cur:
                clo, chi = _box(c)
                if np.all(lo < chi - 1e-12) and np.all(clo < hi - 1e-12):
                    assert abs(_level(b) - _level(c)) <= 1
        if [tuple(_box(b)[0]) + (_level(b),) for b in out] == [tuple(_box(b)[0]) + (_level(b),) for b in cur]:
            return out
        cur = out
    return cur


def _in_corner(b):
    return bool(np.all(_box(b)[1] <= 0.25 + 1e-12))


def test_single_target_nests_and_tiles():
    tree = W.flat_box_tree(base=(4, 4, 4), n=4, refine=())
    out = _adapt_until_stable(_blocks(tree), lambda b: 3 if _in_corner(b) else 0)
    _check_tree(out)
    lv = [_level(b) for b in out]
    assert max(lv) == 3
    # the target region is entirely at level 3
    fine = [b for b in out if _level(b) == 3]
    assert abs(sum(float(np.prod(_box(b)[1] - _box(b)[0])) for b in fine) - 0.25 ** 3) < 1e-12
    assert all(_in_corner(b) for b in fine)
    # a base block far from it (opposite corner region, two blocks away) stays at level 0
    far = [b for b in out if np.allclose(_box(b)[0], (0.5, 0.5, 0.5))]
    assert len(far) == 1 and _level(far[0]) == 0
    # interior faces are block faces, lat = finest level - level
    for b in out:
        assert list(b.bc) == [hamr.BC_BLOCK] * 6 or any(x == 1 for x in b.bc)
        assert b.lat == 3 - _level(b)


def test_derefines_when_the_targets_drop():
    tree = W.flat_box_tree(base=(4, 4, 4), n=4, refine=())
    cur = _blocks(tree)
    mid = _adapt_until_stable(cur, lambda b: 2 if np.allclose(_box(b)[0] // 0.25, (1, 1, 1)) else 0)
    assert len(mid) > len(cur) and max(_level(b) for b in mid) == 2
    back = _adapt_until_stable(mid, lambda b: 0)
    assert len(back) == len(cur) and all(_level(b) == 0 for b in back)
    _check_tree(back)


def test_moving_target_and_bad_inputs():
    tree = W.flat_box_tree(base=(4, 4, 4), n=4, refine=())
    cur = _blocks(tree)
    rng = np.random.default_rng(3)
    for _ in range(3):
        target = list(rng.integers(0, 3, size=len(cur)) * (rng.random(len(cur)) < 0.1))
        cur = hamr.tree_adapt(cur, target, (0, 0, 0), (0.25, 0.25, 0.25))
        _check_tree(cur)
    # overlapping blocks are refused
    bad = _blocks(tree) + _blocks(tree)[:1]
    with pytest.raises(hamr.HamrError):
        hamr.tree_adapt(bad, [0] * len(bad), (0, 0, 0), (0.25, 0.25, 0.25))


# ---- spherical grids with polar axes (hamr_tree_adapt_polar; Sec. 3.3.1): 6-way splits on the axis

def _dicts(out):
    return [dict(n1=b.n1, n2=b.n2, n3=b.n3, x1min=b.x1min, x2min=b.x2min, x3min=b.x3min, dx1=b.dx1, dx2=b.dx2,
                 dx3=b.dx3, bc=list(b.bc), lat=b.lat) for b in out]


def _polar_base():
    import math
    base = W.c3_blocks(nb=(4, 4, 2), n=8, disk=set(), level2=set(), polar_split=[])
    x1a, x1b = math.log(1.2), math.log(50.0)
    return base, (x1a, 0.0, 0.0), ((x1b - x1a) / 4, math.pi / 4, math.pi)


def _covers(blocks, volume):
    vol = sum(b["n1"] * b["dx1"] * b["n2"] * b["dx2"] * b["n3"] * b["dx3"] for b in blocks)
    assert abs(vol - volume) <= 1e-9 * volume


def test_polar_blocks_split_six_way_and_merge_back():
    import math
    base, dlo, ext = _polar_base()
    volume = (math.log(50.0) - math.log(1.2)) * math.pi * 2 * math.pi
    # refine the polar blocks at r index 1: each splits into 2 axis children and 4 off-axis children
    tgt = [1 if (b["group"] == "polar base" and abs(b["x1min"] - (dlo[0] + ext[0])) < 1e-9) else 0 for b in base]
    out = _dicts(hamr.tree_adapt(_blocks(base), tgt, dlo, ext, periodic=(0, 0, 1), axis=(1, 1)))
    _covers(out, volume)
    assert not W.nesting_violations(out)
    axis_kids = [b for b in out if b["dx1"] < ext[0] / 8 * 0.75 and b["n3"] * b["dx3"] > 0.99 * ext[2]]
    far_kids = [b for b in out if b["dx1"] < ext[0] / 8 * 0.75 and b["n3"] * b["dx3"] < 0.51 * ext[2]]
    # 4 refined polar base blocks (2 poles x 2 in phi): 2 axis + 4 off-axis children each
    assert len(axis_kids) == 8 and len(far_kids) == 16, (len(axis_kids), len(far_kids))
    for b in axis_kids:
        assert b["n3"] == 4 and (b["x2min"] == 0.0 or abs(b["x2min"] + b["n2"] * b["dx2"] - math.pi) < 1e-9)
    # every region moved by at most a factor 2 in every direction; targets back to 0 merge the children
    back = _dicts(hamr.tree_adapt(_blocks(out), [0] * len(out), dlo, ext, periodic=(0, 0, 1), axis=(1, 1)))
    assert len(back) == len(base)
    for b, c in zip(sorted(back, key=lambda b: (b["x3min"], b["x2min"], b["x1min"])),
                    sorted(base, key=lambda b: (b["x3min"], b["x2min"], b["x1min"]))):
        for k in ("n1", "n2", "n3", "x1min", "x2min", "x3min", "dx1", "dx2", "dx3"):
            assert abs(b[k] - c[k]) <= 1e-12 * max(1.0, abs(c[k])), k


def test_polar_refinement_nests_in_every_direction():
    """Two levels on an axis child: the tree grows 6-way splits on the axis, octree splits elsewhere, and
    refines neighbours until no face or edge neighbours are more than a factor 2 apart in x1, x2 or x3
    (the axis children's x3 cells are the wide ones)."""
    import math
    base, dlo, ext = _polar_base()
    volume = (math.log(50.0) - math.log(1.2)) * math.pi * 2 * math.pi
    cur = base
    for _ in range(3):
        tgt = []
        for b in cur:
            near = (b["x2min"] == 0.0 and b["x3min"] == 0.0 and b["x1min"] < dlo[0] + 2.01 * ext[0]
                    and b["x1min"] >= dlo[0] + 0.99 * ext[0])
            tgt.append(2 if near else 0)
        cur = _dicts(hamr.tree_adapt(_blocks(cur), tgt, dlo, ext, periodic=(0, 0, 1), axis=(1, 1)))
        _covers(cur, volume)
        assert not W.nesting_violations(cur)
    levels = {int(round(math.log2(ext[0] / (b["n1"] * b["dx1"])))) for b in cur}
    assert levels == {0, 1, 2}, levels
    # level-2 blocks on the axis keep the base polar rows' x3 cells; octree descendants halve them
    on_axis = [b for b in cur if b["x2min"] == 0.0 and b["dx1"] < ext[0] / 8 / 3]
    assert on_axis and all(abs(b["dx3"] - ext[2] / 4) < 1e-12 for b in on_axis)
