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
