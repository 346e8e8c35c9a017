"""All options of the step together on the torus block (upwinded EMFs, the
PPM shock flattener, the Aitken inversion, drift-frame floors, two levels of
internal SMR), against the oracle with the same options: the FP64 path at the
FP64 bars, the mixed-precision path at the mixed bars of the plain torus
(tests/test_gpu_mixed.py), div B at round-off in both. One exception,
measured: with drift-frame floors the mixed path's velocity error after ten
steps is 8e-5 (1.2e-4 with every option) instead of 3e-6: the floored,
magnetised atmosphere re-inverts a mixture whose velocity follows the ratio
of the cell's own momentum to the added material, and the FP32 edge values
shift that ratio; the velocity bar of that case is 5e-4. The FP64 path with
every option stays at round-off (1e-13)."""
import numpy as np
import pytest

import oracle as O

from helpers import face_interior, gpu_grid, interior, rel_l1, torus_case
from test_gpu_mixed import div_b, errors, torus_bars

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
OPTS = dict(emf=1, flatten=1, inversion=1, floor_frame=1, smr=2)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _case():
    geo, d, prim, bf = torus_case(64, 32, 16, seed=1912)
    for k, v in OPTS.items():
        setattr(d, k, v)
    return d, prim, bf


@pytest.mark.parametrize("precision,nsteps", [(0, 1), (0, 10), (1, 1), (1, 10)])
def test_all_options_against_oracle(precision, nsteps):
    from paper_1912_10192_gb300 import hamr
    d, prim, bf = _case()
    b = hamr.block(d.n1, d.n2, d.n3, d.x1min, d.x2min, d.x3min, d.dx1, d.dx2, d.dx3, tuple(d.bc))
    g = hamr.Grid([b], metric=d.metric, a=d.a, gam=d.gam, cour=d.cour, floors=d.floors, precision=precision,
                  **OPTS)
    g.set_state(torch.from_numpy(prim).cuda(), torch.from_numpy(bf).cuda())
    og = O.Grid(d)
    og.set(prim, bf)
    for _ in range(nsteps):
        st = g.step(stats=True)
        og.step(st["dt_used"])
    p, bb = g.get_state()
    po, bo = og.get()
    g.close()
    e = errors(d, p, bb, po, bo)
    print("all options, precision %d, %d steps:" % (precision, nsteps), e)
    if precision == 0:
        bar = {k: (1e-12 if nsteps == 1 else 1e-9) for k in e}
    else:
        bar = torus_bars(nsteps)
        bar["utilde"] = max(bar["utilde"], 5e-4)
    for k, v in e.items():
        assert v <= bar[k], (k, v, e)
    assert div_b(d, bb) <= max(4.0 * div_b(d, bo), 1e-14)
