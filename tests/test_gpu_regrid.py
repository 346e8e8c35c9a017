"""Dynamic refinement on the GPU (Sec. 3.2): hamr_grid_regrid against the
oracle's regridding (copy, restriction, MINMOD and Balsara prolongation) on
flat boxes and a Kerr-Schild torus tree, the per-block criterion input
(hamr_grid_block_max), and an adaptive run in which the refined region
follows an advected dense blob while the face field stays divergence-free."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

NG = 3
pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def ora_blocks(blocks):
    return [O.make_block(b["n1"], b["n2"], b["n3"], b["x1min"], b["x2min"], b["x3min"], b["dx1"], b["dx2"],
                         b["dx3"], b["bc"], b["lat"]) for b in blocks]


def pair(blocks, states, phys, **kw):
    from paper_1912_10192_gb300 import hamr
    a = O.AmrGrid(phys, ora_blocks(blocks))
    g = hamr.Grid([hamr.block_from_dict(b) for b in blocks], metric=phys.metric, a=phys.a, gam=phys.gam,
                  cour=phys.cour, floors=phys.floors, **kw)
    for i, (p, bf) in enumerate(states):
        a.set(i, p, bf)
        g.set_state(p, bf, block=i)
    return a, g


def compare(a, g, blocks, bar):
    worst = 0.0
    for i, b in enumerate(blocks):
        pg, bg = g.get_state(block=i)
        po, bo = a.get(i)
        s = (slice(NG, NG + b["n3"]), slice(NG, NG + b["n2"]), slice(NG, NG + b["n1"]))
        sc = np.abs(po[(slice(0, 5),) + s]).max()
        worst = max(worst, np.abs(pg[(slice(0, 5),) + s] - po[(slice(0, 5),) + s]).max() / sc)
        fs = [(slice(NG, NG + b["n3"]), slice(NG, NG + b["n2"]), slice(NG, NG + b["n1"] + 1)),
              (slice(NG, NG + b["n3"]), slice(NG, NG + b["n2"] + 1), slice(NG, NG + b["n1"])),
              (slice(NG, NG + b["n3"] + 1), slice(NG, NG + b["n2"]), slice(NG, NG + b["n1"]))]
        bs = max(np.abs(bo).max(), 1e-300)
        for m in range(3):
            worst = max(worst, np.abs(bg[m][fs[m]] - bo[m][fs[m]]).max() / bs)
    assert worst <= bar, worst
    return worst


def div_b_max(g, blocks):
    out = 0.0
    for i, b in enumerate(blocks):
        _, bf = g.get_state(block=i)
        n1, n2, n3 = b["n1"], b["n2"], b["n3"]
        f1 = bf[0][NG:NG + n3, NG:NG + n2, NG:NG + n1 + 1]
        f2 = bf[1][NG:NG + n3, NG:NG + n2 + 1, NG:NG + n1]
        f3 = bf[2][NG:NG + n3 + 1, NG:NG + n2, NG:NG + n1]
        d = np.diff(f1, axis=2) / b["dx1"] + np.diff(f2, axis=1) / b["dx2"] + np.diff(f3, axis=0) / b["dx3"]
        out = max(out, np.abs(d).max() * b["dx1"] / max(np.abs(bf).max(), 1e-300))
    return out


FLAT = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_MINKOWSKI, gam=5.0 / 3.0, cour=0.5, floors=0)


def _as_dicts(descs):
    return [dict(n1=b.n1, n2=b.n2, n3=b.n3, x1min=b.x1min, x2min=b.x2min, x3min=b.x3min, dx1=b.dx1, dx2=b.dx2,
                 dx3=b.dx3, bc=list(b.bc), lat=b.lat) for b in descs]


@pytest.mark.parametrize("src,dst", [((), ((1, 1, 0),)), (((0, 1, 1),), ()), (((0, 0, 0),), ((1, 1, 1),)),
                                     (((0, 0, 0),), ((0, 0, 0), (1, 0, 0)))])
def test_regrid_parity_flat_box(src, dst):
    from paper_1912_10192_gb300 import hamr
    old = W.flat_box_tree(base=(2, 2, 2), n=6, refine=src)
    new = W.flat_box_tree(base=(2, 2, 2), n=6, refine=dst)
    a, g = pair(old, W.flat_box_state(old, bamp=0.2), FLAT)
    if len(old) > 1:
        a.period()
        g.batch_step(2 ** max(b["lat"] for b in old))
    a2 = a.regrid(ora_blocks(new))
    g.regrid([hamr.block_from_dict(b) for b in new])
    compare(a2, g, new, 1e-12)
    assert div_b_max(g, new) < 1e-13
    g.close()


@pytest.mark.parametrize("src,dst", [
    (dict(), dict(split=((1, 0, 1),))),                                     # 6-way split of a coarse block
    (dict(split=((0, 1, 0),)), dict(split=())),                             # the 6 children merged back
    (dict(refine=((0, 0, 0),), split=()), dict(refine=((0, 0, 0),), split=((1, 0, 0),))),  # next to finer blocks
    (dict(split=((0, 0, 0),)), dict(refine=((0, 0, 0),), split=())),      # axis children refined in x3 only
    (dict(refine=((0, 0, 0),), split=()), dict(split=((0, 0, 0),))),      # octants merged in x3 only
    (dict(split=((0, 1, 0),)), dict(split=((0, 0, 0),)))])                 # a split next to a merge
def test_regrid_parity_flat_box_six_way(src, dst):
    """6-way splits (workloads.split6: two children keep the parent's x3 cells, 2 x 2 x 1 fine cells per
    coarse cell; four halve all widths) and their merge, against the oracle's regridding."""
    from paper_1912_10192_gb300 import hamr
    old = W.flat_box_tree6(base=(2, 2, 2), n=6, **src)
    new = W.flat_box_tree6(base=(2, 2, 2), n=6, **dst)
    a, g = pair(old, W.flat_box_state(old, bamp=0.2), FLAT)
    if len(old) > 1:
        a.period()
        g.batch_step(2 ** max(b["lat"] for b in old))
    a2 = a.regrid(ora_blocks(new))
    g.regrid([hamr.block_from_dict(b) for b in new])
    compare(a2, g, new, 1e-12)
    assert div_b_max(g, new) < 1e-13
    g.close()


def test_regrid_parity_torus_polar_split():
    """The polar blocks of a Kerr-Schild torus tree split 6-way at run time and merged again (the C3
    tree's polar rule, here as a regrid), against the oracle."""
    from paper_1912_10192_gb300 import hamr
    KS = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=13.0 / 9.0, cour=0.8)
    old = W.c3_blocks(nb=(3, 4, 2), n=8, disk=set(), level2=set(), polar_split=[])
    new = W.c3_blocks(nb=(3, 4, 2), n=8, disk=set(), level2=set(), polar_split=[1])
    assert not W.nesting_violations(new)
    for bl in (old, new):
        for b in bl:
            b["lat"] = 0
    a, g = pair(old, W.torus_blocks(old, seed=3), KS)
    a2 = a.regrid(ora_blocks(new))
    g.regrid([hamr.block_from_dict(b) for b in new])
    compare(a2, g, new, 1e-12)
    assert div_b_max(g, new) < 1e-12   # the oracle's own: 1e-13 of max |Bbar| / dx1
    a3 = a2.regrid(ora_blocks(old))
    g.regrid([hamr.block_from_dict(b) for b in old])
    compare(a3, g, old, 1e-12)
    g.close()


def test_adaptive_polar_refinement_matches_oracle():
    """hamr_tree_adapt_polar marks the polar blocks at r index 1 of a torus tree for level 1 (6-way splits
    on both axes), the GPU and the oracle regrid onto that tree and take one LAT period (levels 0 and 1)."""
    import math
    from paper_1912_10192_gb300 import hamr
    KS = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=13.0 / 9.0, cour=0.8)
    old = W.c3_blocks(nb=(3, 4, 2), n=8, disk=set(), level2=set(), polar_split=[])
    for b in old:
        b["lat"] = 0
    x1a, x1b = math.log(1.2), math.log(50.0)
    dlo, ext = (x1a, 0.0, 0.0), ((x1b - x1a) / 3, math.pi / 4, math.pi)
    tgt = [1 if (b["group"] == "polar base" and abs(b["x1min"] - (x1a + ext[0])) < 1e-9) else 0 for b in old]
    new = hamr.tree_adapt([hamr.block_from_dict(b) for b in old], tgt, dlo, ext, periodic=(0, 0, 1), axis=(1, 1))
    new = _as_dicts(new)
    assert len(new) == len(old) + 4 * 5 and not W.nesting_violations(new)
    a, g = pair(old, W.torus_blocks(old, seed=3), KS)
    a2 = a.regrid(ora_blocks(new))
    g.regrid([hamr.block_from_dict(b) for b in new])
    compare(a2, g, new, 1e-12)
    lmax = max(b["lat"] for b in new)
    assert lmax == 1
    a2.period()
    g.batch_step(2 ** lmax)
    compare(a2, g, new, 1e-10)
    g.close()


def test_regrid_parity_torus_tree():
    from paper_1912_10192_gb300 import hamr
    KS = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=13.0 / 9.0, cour=0.8)
    old = W.torus_tree(nb=(4, 2, 2), n=(8, 8, 8), refine=[(1, 0, 0)])
    new = W.torus_tree(nb=(4, 2, 2), n=(8, 8, 8), refine=[(2, 1, 1), (2, 0, 1)])
    a, g = pair(old, W.torus_blocks(old, seed=3), KS)
    a2 = a.regrid(ora_blocks(new))
    g.regrid([hamr.block_from_dict(b) for b in new])
    compare(a2, g, new, 1e-12)
    g.close()


def test_block_max_and_adaptive_blob():
    """A dense blob advected diagonally through a periodic box of 4^3 base blocks: every period the
    blocks whose maximum density exceeds 1.5 are marked for level 2, hamr_tree_adapt nests the tree and
    hamr_grid_regrid moves the state; the blob's block stays at level 2 and div B at round-off."""
    from paper_1912_10192_gb300 import hamr
    base = W.flat_box_tree(base=(4, 4, 4), n=8, refine=())
    states = []
    v = np.array([0.3, 0.2, 0.1])
    lor = 1.0 / math.sqrt(1.0 - v @ v)
    for st, b in zip(W.flat_box_state(base, amp=0.0, bamp=0.02), base):
        p, bf = st
        x = b["x1min"] + (np.arange(-NG, b["n1"] + NG) + 0.5) * b["dx1"]
        y = b["x2min"] + (np.arange(-NG, b["n2"] + NG) + 0.5) * b["dx2"]
        z = b["x3min"] + (np.arange(-NG, b["n3"] + NG) + 0.5) * b["dx3"]
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        r2 = (X - 0.3) ** 2 + (Y - 0.3) ** 2 + (Z - 0.3) ** 2
        p[0] = 1.0 + 2.0 * np.exp(-r2 / 0.01)
        p[1] = 1.0
        p[2:5] = (lor * v)[:, None, None, None]
        states.append((p, bf))
    g = hamr.Grid([hamr.block_from_dict(b) for b in base], metric=hamr.METRIC_MINKOWSKI, gam=5.0 / 3.0, cour=0.4,
                  floors=0)
    for i, (p, bf) in enumerate(states):
        g.set_state(p, bf, block=i)
    blocks = [hamr.block_from_dict(b) for b in base]
    regrids = 0
    for it in range(6):
        for _ in range(3):  # one level per adaptation: repeat until the tree is stable
            mx = g.block_max(0)
            host = max(g.get_state(block=i)[0][0][NG:-NG, NG:-NG, NG:-NG].max() for i in range(len(blocks)))
            assert abs(mx.max() - host) <= 1e-15 * host
            target = [2 if m > 1.5 else 0 for m in mx]
            new = hamr.tree_adapt(blocks, target, (0, 0, 0), (0.25, 0.25, 0.25))
            if [(b.x1min, b.x2min, b.x3min, b.dx1) for b in new] == [(b.x1min, b.x2min, b.x3min, b.dx1) for b in blocks]:
                break
            blocks = new
            g.regrid(blocks)
            regrids += 1
            assert div_b_max(g, _as_dicts(blocks)) < 1e-12, it
        for _ in range(2):
            g.batch_step(2 ** max(b.lat for b in blocks))
        assert div_b_max(g, _as_dicts(blocks)) < 1e-12, it
    # the densest block is at level 2
    mx = g.block_max(0)
    top = blocks[int(np.argmax(mx))]
    assert abs(top.n1 * top.dx1 - 0.0625) < 1e-12
    levels = [int(round(math.log2(0.25 / (b.n1 * b.dx1)))) for b in blocks]
    print("adaptive blob: %d blocks, levels %s, %d regrids" % (len(blocks), np.bincount(levels).tolist(), regrids))
    g.close()
