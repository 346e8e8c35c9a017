"""Internal SMR on the GPU (Sec. 3.3.2, the phi-averaging of polar rows)
against the oracle: the torus block with a field threading the poles at the
FP64 bars (1 and 10 steps), groups identical cell by cell, the larger CFL step
where the pole limits it; inside the batched block tree: the torus cut into
same-level blocks and a refined polar block on a faster LAT level (edge
synchronisation and refluxing through grouped rows), one period each against
the oracle."""
import numpy as np
import pytest

import oracle as O

from helpers import (NG, face_interior, gpu_grid, interior, ora_tree, polar_field, polar_field_desc,
                     refined_polar_tree, rel_l1, torus_case, tree_errors)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("nsteps,bar", [(1, 1e-12), (10, 1e-9)])
def test_smr_torus_parity(nsteps, bar):
    geo, d, prim, bf = torus_case(64, 32, 16, seed=1912)
    d.smr = 2
    polar_field_desc(bf, d, B0=1e-4)  # the grouped rows' EMFs are then not zero
    g = gpu_grid(d)
    g.set_state(_cu(prim), _cu(bf))
    og = O.Grid(d)
    og.set(prim, bf)
    for _ in range(nsteps):
        st = g.step(stats=True)
        dto = og.step()
    pg, bg = g.get_state()
    po, bo = og.get()
    g.close()
    assert abs(st["dt_used"] - dto) <= 1e-12 * dto
    errs = {"rho": rel_l1(interior(pg[0], d), interior(po[0], d)),
            "u": rel_l1(interior(pg[1], d), interior(po[1], d)),
            "utilde": (sum(np.abs(interior(pg[v], d) - interior(po[v], d)).sum() for v in (2, 3, 4))
                       / sum(np.abs(interior(po[v], d)).sum() for v in (2, 3, 4)))}
    fg, fo = face_interior(bg, d), face_interior(bo, d)
    errs["Bface"] = sum(np.abs(x - y).sum() for x, y in zip(fg, fo)) / sum(np.abs(y).sum() for y in fo)
    for k, e in errs.items():
        assert e <= bar, (k, e, errs)
    # groups of the rows next to the poles are single cells on the GPU too
    for j, w in ((0, 4), (1, 2), (d.n2 - 1, 4), (d.n2 - 2, 2)):
        row = pg[:5, NG:NG + d.n3, NG + j, NG:NG + d.n1].reshape(5, d.n3 // w, w, d.n1)
        assert np.abs(row - row[:, :, :1, :]).max() == 0.0, (j, w)


def test_smr_time_step_gain():
    dts = []
    for smr in (0, 2):
        geo, d, prim, bf = torus_case(64, 32, 64, seed=1912)
        d.smr = smr
        g = gpu_grid(d)
        g.set_state(_cu(prim), _cu(bf))
        dts.append(g.step(stats=True)["dt_next"])
        g.close()
    print("CFL step without / with internal SMR (2 levels): %.4g / %.4g" % tuple(dts))
    assert dts[1] > 1.3 * dts[0], dts  # measured 1.43 (the rate also has the x1 and x2 terms)


def _tree_grid(blocks, states, **kw):
    from paper_1912_10192_gb300 import hamr
    g = hamr.Grid([hamr.block_from_dict(b) for b in blocks], **kw)
    for i, (p, bf) in enumerate(states):
        g.set_state(p, bf, block=i)
    return g


def test_smr_split_torus_tree_parity():
    """The torus with a field through the poles cut into 2 x 2 x 2 same-level blocks, two SMR levels:
    two periods of the batched path against the oracle's block tree."""
    geo, d, prim, bf = torus_case(32, 32, 16, seed=3)
    polar_field_desc(bf, d, B0=1e-4)
    n = (16, 16, 8)
    blocks, states = [], []
    for kb in range(2):
        for jb in range(2):
            for ib in range(2):
                bc = [4] * 6
                bc[ib] = O.BC_OUTFLOW_NOINFLOW
                bc[2 + jb] = O.BC_POLAR
                bc[4 + kb] = O.BC_PERIODIC
                i0, j0, k0 = ib * n[0], jb * n[1], kb * n[2]
                blocks.append(dict(n1=n[0], n2=n[1], n3=n[2], x1min=d.x1min + i0 * d.dx1,
                                   x2min=d.x2min + j0 * d.dx2, x3min=d.x3min + k0 * d.dx3, dx1=d.dx1, dx2=d.dx2,
                                   dx3=d.dx3, bc=bc, lat=0))
                pb = np.zeros((8, n[2] + 6, n[1] + 6, n[0] + 6))
                bb = np.zeros((3, n[2] + 6, n[1] + 6, n[0] + 6))
                pb[:, 3:3 + n[2], 3:3 + n[1], 3:3 + n[0]] = prim[:, 3 + k0:3 + k0 + n[2], 3 + j0:3 + j0 + n[1],
                                                                  3 + i0:3 + i0 + n[0]]
                bb[:, 3:4 + n[2], 3:4 + n[1], 3:4 + n[0]] = bf[:, 3 + k0:4 + k0 + n[2], 3 + j0:4 + j0 + n[1],
                                                                3 + i0:4 + i0 + n[0]]
                states.append((pb, bb))
    d.smr = 2
    a = ora_tree(d, blocks, states)
    g = _tree_grid(blocks, states, metric=d.metric, a=d.a, gam=d.gam, cour=d.cour, floors=d.floors, smr=2)
    for _ in range(2):
        a.period()
        g.batch_step(1)
    errs = tree_errors(g, a, blocks)
    g.close()
    for k, e in errs.items():
        assert e <= 1e-10, (k, e, errs)


def test_smr_refined_polar_tree_parity():
    """A polar block split 6-way next to coarser polar blocks on a slower LAT level, an explosion over
    the axis across the refluxed face, one SMR level: three periods of the batched path (grouped EMFs
    after the edge synchronisation, grouped refluxed cells) against the oracle."""
    blocks, states = refined_polar_tree()
    phys = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_SPHERICAL, gam=5.0 / 3.0, cour=0.8, floors=0,
                       smr=1)
    a = ora_tree(phys, blocks, states)
    g = _tree_grid(blocks, states, metric=O.METRIC_SPHERICAL, gam=5.0 / 3.0, cour=0.8, floors=0, smr=1)
    lmax = max(b["lat"] for b in blocks)
    for _ in range(3):
        a.period()
        g.batch_step(2 ** lmax)
    errs = tree_errors(g, a, blocks)
    g.close()
    for k, e in errs.items():
        assert e <= 1e-10, (k, e, errs)


@pytest.mark.parametrize("precision", [0, 1])
def test_c3_tree_with_internal_smr(precision):
    """The 512-block C3 tree (13.1 M cells) with two internal SMR levels in its polar rows, one LAT
    period from the torus state: the CFL fine step grows over the same tree without SMR from the limit
    of the polar base blocks' first rows (phi term) to that of the radial term in the innermost cells,
    inside the horizon, of the equatorial base blocks: 0.01359 -> 0.02000 (1.47x; the oracle's
    characteristic speeds on the same state give both figures), at most 1e-4 of the inversions fail,
    and every polar block keeps div B at round-off."""
    from paper_1912_10192_gb300 import hamr
    from paper_1912_10192_gb300 import workloads as W
    dts = {}
    for smr in (0, 2):
        blocks = W.c3_tree(n=32, smr=smr)
        states = W.torus_blocks(blocks, seed=3)
        g = hamr.Grid([hamr.block_from_dict(b) for b in blocks], precision=precision, smr=smr)
        for i, (p, bf) in enumerate(states):
            g.set_state(p, bf, block=i)
        del states
        st = g.batch_step(8, stats=True)
        dts[smr] = st["dt_used"]
        assert st["dt_used"] > 0 and st["c2p_fail"] <= 1e-4 * st["c2p_ok"], st
        if smr:
            for i, b in enumerate(blocks):
                if 2 not in (b["bc"][2], b["bc"][3]):
                    continue
                p, bf = g.get_state(block=i)
                assert np.isfinite(p).all()
                n1, n2, n3, s = b["n1"], b["n2"], b["n3"], NG
                div = ((bf[0][s:s + n3, s:s + n2, s + 1:s + n1 + 1] - bf[0][s:s + n3, s:s + n2, s:s + n1]) / b["dx1"]
                       + (bf[1][s:s + n3, s + 1:s + n2 + 1, s:s + n1] - bf[1][s:s + n3, s:s + n2, s:s + n1]) / b["dx2"]
                       + (bf[2][s + 1:s + n3 + 1, s:s + n2, s:s + n1] - bf[2][s:s + n3, s:s + n2, s:s + n1]) / b["dx3"])
                scale = np.abs(bf).max() / min(b["dx1"], b["dx2"], b["dx3"])
                assert np.abs(div).max() <= 1e-12 * scale, i
        g.close()
    assert 1.4 * dts[0] < dts[2] < 1.55 * dts[0], dts
