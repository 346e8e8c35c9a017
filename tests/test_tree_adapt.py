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
