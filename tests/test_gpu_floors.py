"""Floors in the drift frame on the GPU (Sec. 2.7, after Ressler et al.
2017) against the oracle: the torus block, whose magnetised atmosphere is
floored every step, and a refined tree, at the FP64 bars; and over a longer
run, what the drift frame is for: fluid-frame injection keeps the Lorentz
factor of the floored funnel flow, the drift frame lets the added mass slow
it."""
import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

from helpers import face_interior, gpu_grid, interior, rel_l1, torus_case

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


def errors(d, pg, bg, po, bo):
    e = {"rho": rel_l1(interior(pg[0], d), interior(po[0], d)),
         "u": rel_l1(interior(pg[1], d), interior(po[1], d)),
         "utilde": (sum(np.abs(interior(pg[v], d) - interior(po[v], d)).sum() for v in (2, 3, 4))
                    / sum(np.abs(interior(po[v], d)).sum() for v in (2, 3, 4)))}
    fg, fo = face_interior(bg, d), face_interior(bo, d)
    e["Bface"] = sum(np.abs(x - y).sum() for x, y in zip(fg, fo)) / sum(np.abs(y).sum() for y in fo)
    return e


@pytest.mark.parametrize("nsteps,bar", [(1, 1e-12), (10, 1e-9)])
def test_drift_floor_torus_parity(nsteps, bar):
    geo, d, prim, bf = torus_case(64, 32, 16, seed=1912)
    d.floor_frame = O.FLOOR_DRIFT
    g = gpu_grid(d)
    g.set_state(_cu(prim), _cu(bf))
    og = O.Grid(d)
    og.set(prim, bf)
    for _ in range(nsteps):
        st = g.step(stats=True)
        og.step()
    pg, bg = g.get_state()
    po, bo = og.get()
    g.close()
    print("drift floors, %d steps: floor hits %d" % (nsteps, st["floor_hits"]))
    errs = errors(d, pg, bg, po, bo)
    for k, e in errs.items():
        assert e <= bar, (k, e, errs)


def test_drift_floor_tree_parity():
    from test_gpu_amr import KS, field_errors, run_pair
    blocks = W.torus_tree(nb=(4, 2, 2), n=(8, 8, 8), refine=[(1, 0, 0), (2, 1, 1)], lat_base=1, lat_refined=0)
    states = W.torus_blocks(blocks, seed=3)
    phys = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, floor_frame=O.FLOOR_DRIFT, **KS)
    out, dts = run_pair(blocks, states, phys, 1, floor_frame=1)
    errs = field_errors(blocks, out)
    for k, e in errs.items():
        assert e <= 1e-11, (k, e, errs)


def test_drift_frame_slows_the_floored_funnel():
    """200 steps of the 64x32x16 torus in each frame: Lorentz factors of the floored cells."""
    from paper_1912_10192_gb300 import hamr
    res = {}
    for frame in (hamr.FLOOR_FLUID, hamr.FLOOR_DRIFT):
        geo, d, prim, bf = torus_case(64, 32, 16, seed=1912)
        d.floor_frame = frame
        g = gpu_grid(d)
        g.set_state(_cu(prim), _cu(bf))
        for _ in range(200):
            g.step()
        p, _ = g.get_state()
        g.close()
        q = interior(p, d)
        geo_g = np.array([[O.geom(d, geo.x1min + (i + 0.5) * geo.dx1, geo.x2min + (j + 0.5) * geo.dx2)[0][1:, 1:]
                           for i in range(d.n1)] for j in range(d.n2)])  # (n2, n1, 3, 3)
        ut = np.moveaxis(q[2:5], 0, -1)  # (n3, n2, n1, 3)
        qsq = np.einsum("kjia,jiab,kjib->kji", ut, geo_g, ut)
        lor = np.sqrt(1.0 + qsq)
        res[frame] = (lor.max(), (lor > 5).sum(), np.isfinite(q).all())
    print("max Lorentz factor, cells above 5: fluid frame %s, drift frame %s" % (res[0][:2], res[1][:2]))
    assert res[1][2] and res[0][2]
    assert res[1][0] <= res[0][0] * 1.05
