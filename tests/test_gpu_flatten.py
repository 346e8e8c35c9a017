"""The PPM shock flattener on the GPU (Sec. 2.1, Colella & Woodward 1984)
against the oracle: colliding relativistic streams along each direction
(the row kernel along x1, the pencil sweeps along x2 and x3, the per-cell
FP32 kernel), the torus block, a refined tree and the no-allocation step,
at the FP64 bars of the plain path; and on the GPU alone the property the
oracle's pins fix (post-shock overshoot below 2% with the flattener, above
5% without)."""
import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

from helpers import NG, face_interior, gpu_grid, interior, rel_l1, torus_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GAM = 5.0 / 3.0
STREAMS = ((1.0, 0.01, 0.9), (1.0, 0.01, -0.9))  # rho, p, v: cold streams colliding at +-0.9


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def streams_case(n, axis, flatten=1):
    """The colliding streams along x_axis of a flat box (n cells along it, 4 across)."""
    prim, bf = W.riemann_block(n, *STREAMS, gam=GAM)
    if axis == 2:
        prim = np.ascontiguousarray(np.swapaxes(prim, 2, 3)[[0, 1, 3, 2, 4, 5, 6, 7]])
    elif axis == 3:
        prim = np.ascontiguousarray(np.swapaxes(prim, 1, 3)[[0, 1, 3, 4, 2, 5, 6, 7]])
    bf = np.zeros((3,) + prim.shape[1:])
    nn = [4, 4, 4]
    nn[axis - 1] = n
    h = [1.0, 1.0, 1.0]
    h[axis - 1] = 1.0 / n
    bc = [1] * 6
    bc[2 * (axis - 1)] = bc[2 * (axis - 1) + 1] = 0
    d = O.make_desc(*nn, 0.0, 0.0, 0.0, *h, metric=O.METRIC_MINKOWSKI, gam=GAM, cour=0.5, recon=O.RECON_PPM,
                    riemann=O.FLUX_HLL, bc=tuple(bc), floors=0, flatten=flatten)
    return d, prim, bf


def run_both(d, prim, bf, nsteps):
    g = gpu_grid(d)
    g.set_state(torch.from_numpy(prim).cuda(), torch.from_numpy(bf).cuda())
    og = O.Grid(d)
    og.set(prim, bf)
    for _ in range(nsteps):
        g.step()
        og.step()
    pg, bg = g.get_state()
    po, bo = og.get()
    g.close()
    return pg, bg, po, bo


def errors(d, pg, bg, po, bo):
    e = {"rho": rel_l1(interior(pg[0], d), interior(po[0], d)),
         "u": rel_l1(interior(pg[1], d), interior(po[1], d))}
    e["utilde"] = (sum(np.abs(interior(pg[v], d) - interior(po[v], d)).sum() for v in (2, 3, 4))
                   / sum(np.abs(interior(po[v], d)).sum() for v in (2, 3, 4)))
    fg, fo = face_interior(bg, d), face_interior(bo, d)
    den = sum(np.abs(y).sum() for y in fo)
    e["Bface"] = sum(np.abs(x - y).sum() for x, y in zip(fg, fo)) / den if den > 0 else 0.0
    return e


@pytest.mark.parametrize("axis", [1, 2, 3])
def test_flattened_streams_parity_each_direction(axis):
    d, prim, bf = streams_case(96, axis)
    pg, bg, po, bo = run_both(d, prim, bf, 20)
    errs = errors(d, pg, bg, po, bo)
    for k in ("rho", "u", "utilde"):
        assert errs[k] <= 1e-9, (axis, k, errs)


@pytest.mark.parametrize("nsteps,bar", [(1, 1e-12), (10, 1e-9)])
def test_flattened_torus_parity(nsteps, bar):
    geo, d, prim, bf = torus_case(64, 32, 16, seed=1912)
    d.flatten = 1
    pg, bg, po, bo = run_both(d, prim, bf, nsteps)
    errs = errors(d, pg, bg, po, bo)
    for k, e in errs.items():
        assert e <= bar, (k, e, errs)


def _overshoot(prec, flatten, n=200, T=0.4):
    import srhd_exact as X
    from paper_1912_10192_gb300 import hamr
    d, prim, bf = streams_case(n, 1, flatten)
    b = hamr.block(n, 4, 4, 0.0, 0.0, 0.0, 1.0 / n, 1.0, 1.0, tuple(d.bc))
    g = hamr.Grid([b], metric=hamr.METRIC_MINKOWSKI, gam=GAM, cour=0.5, floors=0, precision=prec, flatten=flatten)
    g.set_state(torch.from_numpy(prim).cuda(), torch.from_numpy(bf).cuda())
    t = 0.0
    while t < T - 1e-12:
        st = g.step(stats=True)
        t += st["dt_used"]
        if T - t < st["dt_next"]:
            g.step(T - t)
            t = T
    p, _ = g.get_state()
    g.close()
    pstar = X.solve(X.State(*STREAMS[0], GAM), X.State(*STREAMS[1], GAM))[0]
    return (GAM - 1.0) * p[1][NG + 1, NG + 1, NG:NG + n].max() / pstar


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_flattener_removes_the_overshoot_on_the_gpu(prec):
    from paper_1912_10192_gb300 import hamr
    pr = hamr.PREC_FP64 if prec == "fp64" else hamr.PREC_MIXED
    plain, flat = _overshoot(pr, 0), _overshoot(pr, 1)
    print(prec, "pressure maximum / p*: plain %.4f, flattened %.4f" % (plain, flat))
    assert plain > 1.05 and flat < 1.02, (plain, flat)


def test_flattened_tree_parity():
    """One LAT period of the refined torus tree of the batched-path tests with the flattener."""
    from test_gpu_amr import KS, field_errors, run_pair
    blocks = W.torus_tree(nb=(4, 2, 2), n=(8, 8, 8), refine=[(1, 0, 0), (2, 1, 1)], lat_base=1, lat_refined=0)
    states = W.torus_blocks(blocks, seed=3)
    phys = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, flatten=1, **KS)
    out, dts = run_pair(blocks, states, phys, 1, flatten=1)
    errs = field_errors(blocks, out)
    for k, e in errs.items():
        assert e <= 1e-11, (k, e, errs)


def test_flattened_noalloc_matches_allocating_step():
    from paper_1912_10192_gb300 import hamr
    geo, d, prim, bf = torus_case(16, 8, 8, seed=77)
    d.flatten = 1
    g = gpu_grid(d)
    g.set_state(prim, bf)
    g.step()
    ref = g.get_state()
    tp, tb = torch.from_numpy(prim).cuda(), torch.from_numpy(bf).cuda()
    hamr.block_step_noalloc(g, tp, tb)
    torch.cuda.synchronize()
    errs = errors(d, tp.cpu().numpy(), tb.cpu().numpy(), *ref)
    for k, e in errs.items():
        assert e <= 1e-12, (k, e)
    g.close()
