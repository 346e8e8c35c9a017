"""hamr_block_step_noalloc against hamr_block_step.

The no-allocation step exists for callers that cannot allocate device
memory (a framework that owns the memory pool, or code that must not call
cudaMalloc once it runs); it keeps its scratch in a fixed device array. It
must give the same state as the allocating path, call after call, although
the array keeps the previous call's contents. This file is collected last.
"""
import numpy as np
import pytest

from helpers import face_interior, interior, rel_l1, torus_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _errors(d, pa, ba, pb, bb):
    e = {"rho": rel_l1(interior(pa[0], d), interior(pb[0], d)),
         "u": rel_l1(interior(pa[1], d), interior(pb[1], d))}
    e["utilde"] = (sum(np.abs(interior(pa[v], d) - interior(pb[v], d)).sum() for v in (2, 3, 4))
                   / sum(np.abs(interior(pb[v], d)).sum() for v in (2, 3, 4)))
    fa, fb = face_interior(ba, d), face_interior(bb, d)
    e["Bface"] = sum(np.abs(x - y).sum() for x, y in zip(fa, fb)) / sum(np.abs(y).sum() for y in fb)
    return e


def test_noalloc_matches_allocating_step_two_calls():
    from paper_1912_10192_gb300 import hamr
    from helpers import gpu_grid
    geo, d, prim, bf = torus_case(16, 8, 8, seed=77)
    g = gpu_grid(d)
    g.set_state(prim, bf)
    ref = []
    for _ in range(2):
        g.step()
        ref.append(g.get_state())
    tp = torch.from_numpy(prim).cuda()
    tb = torch.from_numpy(bf).cuda()
    for call in range(2):
        hamr.block_step_noalloc(g, tp, tb)
        torch.cuda.synchronize()
        pa, ba = tp.cpu().numpy(), tb.cpu().numpy()
        errs = _errors(d, pa, ba, *ref[call])
        for k, e in errs.items():
            assert e <= 1e-12, (call, k, e)
    g.close()


def test_noalloc_rejects_blocks_above_its_limit():
    from paper_1912_10192_gb300 import hamr
    from helpers import gpu_grid
    geo, d, prim, bf = torus_case(32, 16, 16, seed=1)
    g = gpu_grid(d)
    tp = torch.from_numpy(prim).cuda()
    tb = torch.from_numpy(bf).cuda()
    with pytest.raises(hamr.HamrError, match="too large for the no-allocation step"):
        hamr.block_step_noalloc(g, tp, tb)
    g.close()


def _flat_box(n, seed):
    """A smooth periodic flat-space state on an n^3 box: sinusoidal density and pressure, a flow and a
    uniform face field (divergence-free)."""
    from paper_1912_10192_gb300 import hamr
    import oracle as O
    rng = np.random.default_rng(seed)
    d = O.make_desc(n, n, n, 0.0, 0.0, 0.0, 1.0 / n, 1.0 / n, 1.0 / n, metric=O.METRIC_MINKOWSKI, gam=5.0 / 3.0,
                    cour=0.5, bc=(hamr.BC_PERIODIC,) * 6, floors=0)
    shp = (n + 6, n + 6, n + 6)
    prim = np.zeros((8,) + shp)
    bf = np.zeros((3,) + shp)
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    s = (slice(3, 3 + n),) * 3
    ph = rng.uniform(0, 2 * np.pi, 4)
    prim[0][s] = 1.0 + 0.3 * np.sin(2 * np.pi * X + ph[0]) * np.cos(2 * np.pi * Y + ph[1])
    prim[1][s] = 1.0 + 0.2 * np.cos(2 * np.pi * Z + ph[2])
    prim[2][s] = 0.3 * np.sin(2 * np.pi * Y + ph[3])
    prim[3][s] = -0.2
    prim[4][s] = 0.1 * np.cos(2 * np.pi * X)
    bf[0][s] = 0.4
    bf[1][s] = -0.3
    bf[2][s] = 0.2
    return d, prim, bf


def _ref_and_noalloc(d, prim, bf, opts):
    from paper_1912_10192_gb300 import hamr
    from helpers import gpu_grid
    for k, v in opts.items():
        setattr(d, k, v)
    g = gpu_grid(d)
    g.set_state(prim, bf)
    g.step()
    ref = g.get_state()
    tp = torch.from_numpy(prim).cuda()
    tb = torch.from_numpy(bf).cuda()
    hamr.block_step_noalloc(g, tp, tb)
    torch.cuda.synchronize()
    g.close()
    return _errors(d, tp.cpu().numpy(), tb.cpu().numpy(), *ref)


def test_noalloc_after_blocks_of_other_shapes():
    """The array keeps the previous call's bytes, laid out with that block's field stride: a block of
    another shape before (the largest accepted, 16^3, then a 6^3 one) must not change the next result,
    with the upwinded EMFs and the shock flattener on (they use scratch fields the plain step leaves
    unused)."""
    for n, seed in ((16, 1), (6, 2)):
        d, prim, bf = _flat_box(n, seed)
        for k, e in _ref_and_noalloc(d, prim, bf, dict(emf=1, flatten=1)).items():
            assert e <= 1e-12, (n, k, e)
    geo, d, prim, bf = torus_case(16, 8, 8, seed=78)
    for k, e in _ref_and_noalloc(d, prim, bf, dict(emf=1, flatten=1)).items():
        assert e <= 1e-12, ("torus", k, e)
    geo, d, prim, bf = torus_case(16, 8, 8, seed=79)
    for k, e in _ref_and_noalloc(d, prim, bf, {}).items():
        assert e <= 1e-12, ("torus plain", k, e)
