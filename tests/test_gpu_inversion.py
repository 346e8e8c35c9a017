"""The Aitken-accelerated inversion on the GPU (Sec. 2.6: the paper's
alternative to the 2-D Newton, after Newman & Hamlin 2014) against the
oracle: standalone inversions of random states from a warm and a cold start,
the torus block and a refined tree at the FP64 bars; and the comparison the
variant exists for (failures and iterations against Newton from the same
starts). Also the mixed-precision form of Newton (FP32 iterations, one FP64
refinement step) against the oracle's FP64 Newton on random states."""
import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

from helpers import face_interior, interior, inversion_bar, rel_l1, torus_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GAM = 13.0 / 9.0


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_invert(U, B, x1, x2, guess, flags, timed=False):
    from paper_1912_10192_gb300 import hamr
    n = len(x1)
    tU, tB, tx1, tx2 = _cu(U.T), _cu(B.T), _cu(x1), _cu(x2)
    tp = _cu(guess.T)
    ts = torch.zeros(n, dtype=torch.int32, device="cuda")
    ti = torch.zeros(n, dtype=torch.int32, device="cuda")
    ms = None
    if timed:  # warm-up, then the timed call on a fresh copy of the guess
        hamr.con2prim(tU, tB, tx1, tx2, tp.clone(), ts, ti, a=0.9375, gam=GAM, flags=flags)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
    hamr.con2prim(tU, tB, tx1, tx2, tp, ts, ti, a=0.9375, gam=GAM, flags=flags)
    if timed:
        e1.record()
    torch.cuda.synchronize()
    if timed:
        ms = e0.elapsed_time(e1)
    return tp.cpu().numpy().T, ts.cpu().numpy(), ti.cpu().numpy(), ms


@pytest.mark.parametrize("start", ["warm", "cold"])
def test_aitken_parity_random_states(start):
    from paper_1912_10192_gb300 import hamr
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=GAM, inversion=O.INV_AITKEN)
    n = 200_000
    prim, x1, x2 = W.random_states(n, seed=23)
    U = O.p2u_many(d, prim, x1, x2)
    guess = prim.copy()
    if start == "warm":
        guess[:, 0] *= 1.05
        guess[:, 1] *= 0.95
        guess[:, 2:5] *= 1.02
    else:
        guess[:, 1] = 1e-3 * guess[:, 0]
        guess[:, 2:5] = 0.0
    po, so, io = O.c2p_many(d, U, prim[:, 5:8], x1, x2, guess)
    pg, sg, ig, _ = gpu_invert(U, prim[:, 5:8], x1, x2, guess, hamr.C2P_AITKEN)
    assert np.array_equal(sg, so)
    ok = so == 0
    assert ok.mean() > 0.999
    # the pressure iteration stops at a tolerance (an extrapolation step below 1e-10 W), not at
    # round-off: its backward error (the relative residual U(p) - U) is bounded like the oracle's
    # (measured over this law: median 2e-14, 99th percentile 3e-11, max 3e-10 on the CPU), and the
    # two results differ by at most the conditioning of the inversion times both residuals
    # (helpers.inversion_bar with the GPU result as p_other)
    pg8 = pg[ok].copy()
    pg8[:, 5:8] = prim[ok, 5:8]
    be = np.abs(O.p2u_many(d, pg8, x1[ok], x2[ok])[:, :5] - U[ok, :5]).sum(axis=1) / np.abs(U[ok, :5]).sum(axis=1)
    assert be.max() < 1e-8 and np.quantile(be, 0.99) < 1e-10, (be.max(), np.quantile(be, 0.99))
    bar = inversion_bar(d, U[ok], prim[ok, 5:8], x1[ok], x2[ok], po[ok], prim[ok], p_other=pg[ok])
    assert np.all(np.abs(pg[ok, :5] - po[ok, :5]) <= bar)
    rel = np.abs(pg[ok, :5] - po[ok, :5]) / np.abs(po[ok, :5]).max(axis=1, keepdims=True)
    assert np.median(rel) < 1e-14 and np.quantile(rel, 0.99) < 1e-11, (np.median(rel), np.quantile(rel, 0.99))
    # the same iteration: map evaluations agree (a cycle more or less where the stopping test is at rounding)
    assert (ig == io).mean() > 0.99 and np.abs(ig - io).max() <= 3


def test_mixed_newton_random_states():
    """The inversion of the mixed-precision cell update (Newton in FP32, then one refinement step with
    the FP64 residuals and the FP32 Jacobian, FP64 Newton where that step is not accepted) on 1M
    states of the wide law from a 5% start: the same outcomes as the oracle's FP64 Newton, results
    within the conditioning bar of both residuals, and a backward error at the FP64 Newton
    tolerance's level (the refinement stops an error of ~1e-7 W at ~1e-14 W for a well-conditioned
    Jacobian; an ill-conditioned one is sent on to FP64 Newton)."""
    from paper_1912_10192_gb300 import hamr
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=GAM)
    n = 1_000_000
    prim, x1, x2 = W.random_states(n, seed=31)
    U = O.p2u_many(d, prim, x1, x2)
    guess = prim.copy()
    guess[:, 0] *= 1.05
    guess[:, 1] *= 0.95
    guess[:, 2:5] *= 1.02
    po, so, io = O.c2p_many(d, U, prim[:, 5:8], x1, x2, guess)
    pg, sg, ig, ms = gpu_invert(U, prim[:, 5:8], x1, x2, guess, hamr.C2P_MIXED, timed=True)
    pn, sn, inn, msn = gpu_invert(U, prim[:, 5:8], x1, x2, guess, 0, timed=True)
    print("mixed Newton: %.2f ms per 1M (FP64 Newton %.2f), iterations %.2f (FP64 %.2f)"
          % (ms, msn, ig[sg == 0].mean(), inn[sn == 0].mean()))
    assert (sg == so).mean() > 0.9999
    ok = (so == 0) & (sg == 0) & (sn == 0)
    assert ok.mean() > 0.999

    def backward(p):  # relative residual |U(p) - U| of each accepted state
        p8 = p[ok].copy()
        p8[:, 5:8] = prim[ok, 5:8]
        return np.abs(O.p2u_many(d, p8, x1[ok], x2[ok])[:, :5] - U[ok, :5]).sum(axis=1) / np.abs(U[ok, :5]).sum(axis=1)

    be, ben = backward(pg), backward(pn)
    print("backward error: mixed median %.1e p99 %.1e max %.1e; FP64 Newton median %.1e p99 %.1e max %.1e"
          % (np.median(be), np.quantile(be, 0.99), be.max(), np.median(ben), np.quantile(ben, 0.99), ben.max()))
    # the tail at the FP64 iteration's level (its tolerance on W, 1e-10, sets both; measured p99 3.4e-11,
    # max 4e-10 for both); the bulk at the refinement's level: the FP32 root's error (~1e-7) times the
    # FP32 Jacobian's relative error and its cancellation (measured median 1.7e-13 against 2.4e-14
    # after the FP64 Newton's last quadratic step)
    assert np.median(be) <= 1e-12
    assert np.quantile(be, 0.99) <= 2.0 * np.quantile(ben, 0.99) + 1e-15 and be.max() <= 2.0 * ben.max() + 1e-15
    bar = inversion_bar(d, U[ok], prim[ok, 5:8], x1[ok], x2[ok], po[ok], prim[ok], p_other=pg[ok])
    assert np.all(np.abs(pg[ok, :5] - po[ok, :5]) <= bar)


def test_aitken_against_newton_from_the_same_starts():
    """Failures and iterations of both energy inversions on 1M states of the wide range, from a warm
    start (5% off) and a cold one (the true rho at rest, u = 1e-3 rho): the pressure iteration converges
    wherever Newton does, and from the cold start also where Newton does not."""
    from paper_1912_10192_gb300 import hamr
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=GAM)
    n = 1_000_000
    prim, x1, x2 = W.random_states(n, seed=6)
    U = O.p2u_many(d, prim, x1, x2)
    rows = []
    for start in ("warm", "cold"):
        guess = prim.copy()
        if start == "warm":
            guess[:, 0] *= 1.05
            guess[:, 1] *= 0.95
            guess[:, 2:5] *= 1.02
        else:
            guess[:, 1] = 1e-3 * guess[:, 0]
            guess[:, 2:5] = 0.0
        res = {}
        for name, flags in (("newton", 0), ("aitken", hamr.C2P_AITKEN)):
            pg, sg, ig, ms = gpu_invert(U, prim[:, 5:8], x1, x2, guess, flags, timed=True)
            ok = sg == 0
            res[name] = ok
            rows.append((start, name, ok.mean(), (sg == 1).mean(), (sg == 2).mean(), ig[ok].mean(), ms))
        assert not np.any(res["newton"] & ~res["aitken"])
        if start == "cold":
            assert res["aitken"].mean() > res["newton"].mean()
    for r in rows:
        print("%s start, %-6s: energy %.4f entropy %.4f failed %.4f, iterations %.2f, %.2f ms per 1M" % r)


@pytest.mark.parametrize("nsteps,bar", [(1, 1e-12), (10, 1e-9)])
def test_aitken_torus_parity(nsteps, bar):
    from helpers import gpu_grid
    geo, d, prim, bf = torus_case(64, 32, 16, seed=1912)
    d.inversion = O.INV_AITKEN
    g = gpu_grid(d)
    g.set_state(_cu(prim), _cu(bf))
    og = O.Grid(d)
    og.set(prim, bf)
    for _ in range(nsteps):
        g.step()
        og.step()
    pg, bg = g.get_state()
    po, bo = og.get()
    g.close()
    errs = {"rho": rel_l1(interior(pg[0], d), interior(po[0], d)),
            "u": rel_l1(interior(pg[1], d), interior(po[1], d)),
            "utilde": (sum(np.abs(interior(pg[v], d) - interior(po[v], d)).sum() for v in (2, 3, 4))
                       / sum(np.abs(interior(po[v], d)).sum() for v in (2, 3, 4)))}
    fg, fo = face_interior(bg, d), face_interior(bo, d)
    errs["Bface"] = sum(np.abs(x - y).sum() for x, y in zip(fg, fo)) / sum(np.abs(y).sum() for y in fo)
    for k, e in errs.items():
        assert e <= bar, (k, e, errs)


def test_aitken_tree_parity():
    """One LAT period of the refined torus tree with the Aitken inversion (cell updates and the
    re-inversion of refluxed cells)."""
    from test_gpu_amr import KS, field_errors, run_pair
    blocks = W.torus_tree(nb=(4, 2, 2), n=(8, 8, 8), refine=[(1, 0, 0), (2, 1, 1)], lat_base=1, lat_refined=0)
    states = W.torus_blocks(blocks, seed=3)
    phys = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, inversion=O.INV_AITKEN, **KS)
    out, dts = run_pair(blocks, states, phys, 1, inversion=1)
    errs = field_errors(blocks, out)
    for k, e in errs.items():
        assert e <= 1e-11, (k, e, errs)
