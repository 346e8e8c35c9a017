"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: relative L1 per field, sum|gpu - oracle| / sum|oracle| over the
interior cells (evolved faces for the staggered field), <= 1e-12 after one
step and <= 1e-9 after ten steps of the torus block, the bar of the FP64
path. The fields are rho, u_g, the velocity utilde^i and the face field
Bbar^i; a vector field is one field (its three components summed together),
and each single component must also stay within 10x the bar. The two codes
contract FMAs and order sums differently, so they agree to rounding, not
bitwise; pure data movement (boundary copies) is compared bitwise.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

from helpers import NG, face_interior, gpu_grid, interior, inversion_bar, rel_l1, torus_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def run_both(d, prim, bf, nsteps, dt=-1.0):
    g = gpu_grid(d)
    g.set_state(torch.from_numpy(prim).cuda(), torch.from_numpy(bf).cuda())
    og = O.Grid(d)
    og.set(prim, bf)
    dts = []
    for _ in range(nsteps):
        st = g.step(dt, stats=True)
        dto = og.step(dt)
        dts.append((st["dt_used"], dto))
    pg, bg = g.get_state()
    po, bo = og.get()
    g.close()
    return pg, bg, po, bo, dts, og


def field_errors(d, pg, bg, po, bo):
    """{field: rel L1} for rho, u_g, the utilde vector, the face-B vector, and each component."""
    errs = {"rho": rel_l1(interior(pg[0], d), interior(po[0], d)),
            "u": rel_l1(interior(pg[1], d), interior(po[1], d))}
    num = sum(np.abs(interior(pg[v], d) - interior(po[v], d)).sum() for v in (2, 3, 4))
    den = sum(np.abs(interior(po[v], d)).sum() for v in (2, 3, 4))
    errs["utilde"] = num / den
    fg, fo = face_interior(bg, d), face_interior(bo, d)
    errs["Bface"] = sum(np.abs(a - b).sum() for a, b in zip(fg, fo)) / sum(np.abs(b).sum() for b in fo)
    comps = {"utilde%d" % (v - 1): rel_l1(interior(pg[v], d), interior(po[v], d)) for v in (2, 3, 4)}
    comps.update({"Bbar%d" % (m + 1): rel_l1(a, b) for m, (a, b) in enumerate(zip(fg, fo)) if np.abs(b).sum() > 0})
    return errs, comps


def assert_parity(errs, comps, bar):
    for k, e in errs.items():
        assert e <= bar, (k, e, errs, comps)
    for k, e in comps.items():
        assert e <= 10 * bar, (k, e, errs, comps)


def test_c2p_parity_random_states():
    from paper_1912_10192_gb300 import hamr
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=13.0 / 9.0)
    n = 200_000
    prim, x1, x2 = W.random_states(n, seed=21)
    U = O.p2u_many(d, prim, x1, x2)
    guess = prim.copy()
    guess[:, 0] *= 1.05
    guess[:, 1] *= 0.95
    guess[:, 2:5] *= 1.02
    po, so, io = O.c2p_many(d, U, prim[:, 5:8], x1, x2, guess)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    tU, tB, tx1, tx2 = cu(U.T), cu(prim[:, 5:8].T), cu(x1), cu(x2)
    tp = cu(guess.T)
    ts = torch.zeros(n, dtype=torch.int32, device="cuda")
    ti = torch.zeros(n, dtype=torch.int32, device="cuda")
    hamr.con2prim(tU, tB, tx1, tx2, tp, ts, ti, a=0.9375, gam=13.0 / 9.0)
    torch.cuda.synchronize()
    pg = tp.cpu().numpy().T
    sg = ts.cpu().numpy()
    # the outcome of every inversion (energy / entropy / failed) is identical
    assert np.array_equal(sg, so)
    ok = so == 0
    # the two results agree to the conditioning of the inversion, state by state
    # (helpers.inversion_bar: |J^-1| of the prim -> cons map times the rounding
    # of evaluating it), and in distribution within the oracle's own spread
    # between two starting points (median 1.8e-15, 99th percentile 7.8e-13,
    # tests/test_inversion_bar.py) with room for a third rounding path
    bar = inversion_bar(d, U[ok], prim[ok, 5:8], x1[ok], x2[ok], po[ok], prim[ok])
    assert np.all(np.abs(pg[ok, :5] - po[ok, :5]) <= bar)
    scale = np.abs(po[ok, :5]).max(axis=1, keepdims=True)
    rel = np.abs(pg[ok, :5] - po[ok, :5]) / scale
    assert np.median(rel) < 1e-14 and np.quantile(rel, 0.99) < 1e-11
    sub = np.nonzero(ok)[0][:20000]
    Ug = O.p2u_many(d, pg[sub], x1[sub], x2[sub])
    Uo = O.p2u_many(d, po[sub], x1[sub], x2[sub])
    den = np.abs(U[sub, :5]).sum(axis=1)
    be_g = np.abs(Ug[:, :5] - U[sub, :5]).sum(axis=1) / den
    be_o = np.abs(Uo[:, :5] - U[sub, :5]).sum(axis=1) / den
    assert be_g.max() < 1e-9 and np.quantile(be_g, 0.99) <= 10 * np.quantile(be_o, 0.99) + 1e-15
    assert np.abs(ti.cpu().numpy() - io).max() <= 1


def test_c2p_entropy_only_and_edge_sizes():
    from paper_1912_10192_gb300 import hamr
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.5, gam=4.0 / 3.0)
    for n in (1, 37, 4099):
        prim, x1, x2 = W.random_states(n, seed=n, a=0.5, lorentz_range=(1, 5), sigma_range=(0, 5))
        U = O.p2u_many(d, prim, x1, x2)
        po, so, _ = O.c2p_many(d, U, prim[:, 5:8], x1, x2, prim, entropy_only=True)
        cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        tp = cu(prim.T)
        ts = torch.zeros(n, dtype=torch.int32, device="cuda")
        hamr.con2prim(cu(U.T), cu(prim[:, 5:8].T), cu(x1), cu(x2), tp, ts, None, a=0.5, gam=4.0 / 3.0,
                      flags=hamr.C2P_ENTROPY_ONLY)
        torch.cuda.synchronize()
        assert np.array_equal(ts.cpu().numpy(), so)
        pg = tp.cpu().numpy().T
        ok = so == 1
        assert np.abs(pg[ok, :5] - po[ok, :5]).max() <= 1e-11 * np.abs(po[ok, :5]).max()


def test_boundaries_bitwise_after_load():
    geo, d, prim, bf = torus_case(16, 8, 8, seed=3)
    g = gpu_grid(d)
    g.set_state(prim, bf)
    pg, bg = g.get_state()
    og = O.Grid(d)
    og.set(prim, bf)
    po, bo = og.get()
    g.close()
    assert np.array_equal(pg[:5], po[:5])
    assert np.array_equal(bg, bo)
    assert np.abs(pg[5:] - po[5:]).max() <= 1e-14 * np.abs(po[5:]).max()


def test_step_parity_torus_64x32x16_one_step():
    geo, d, prim, bf = torus_case(64, 32, 16, seed=1912)
    pg, bg, po, bo, dts, og = run_both(d, prim, bf, 1)
    assert abs(dts[0][0] - dts[0][1]) <= 1e-13 * dts[0][1]
    assert_parity(*field_errors(d, pg, bg, po, bo), 1e-12)


def test_step_parity_torus_64x32x16_ten_steps():
    geo, d, prim, bf = torus_case(64, 32, 16, seed=1912)
    pg, bg, po, bo, dts, og = run_both(d, prim, bf, 10)
    for a, b in dts:
        assert abs(a - b) <= 1e-11 * b
    assert_parity(*field_errors(d, pg, bg, po, bo), 1e-9)


def test_brute_force_8cubed_every_cell():
    """8^3 torus block (coarse, so every cell sees strong gradients) and a flat
    periodic magnetised box: every field of every cell, ghosts included."""
    geo, d, prim, bf = torus_case(8, 8, 8, seed=8)
    pg, bg, po, bo, _, _ = run_both(d, prim, bf, 1)
    for v in range(8):
        scale = np.abs(po[v]).max()
        assert np.abs(pg[v] - po[v]).max() <= 1e-10 * scale, v
    assert np.abs(bg - bo).max() <= 1e-10 * np.abs(bo).max()

    rng = np.random.default_rng(0)
    d2 = O.make_desc(8, 8, 8, 0, 0, 0, 1 / 8, 1 / 8, 1 / 8, metric=O.METRIC_MINKOWSKI, gam=5 / 3, cour=0.5,
                     recon=O.RECON_MC, riemann=O.FLUX_LLF, bc=(1,) * 6, floors=0)
    shp = (14, 14, 14)
    p2 = np.zeros((8,) + shp)
    b2 = np.zeros((3,) + shp)
    s = (slice(3, 11),) * 3
    p2[0][s] = 1 + 0.3 * rng.random((8, 8, 8))
    p2[1][s] = 1 + 0.3 * rng.random((8, 8, 8))
    for v in (2, 3, 4):
        p2[v][s] = 0.3 * rng.standard_normal((8, 8, 8))
    b2[0][s] = 0.3  # uniform field: divergence free
    b2[1][s] = -0.2
    b2[2][s] = 0.1
    pg, bg, po, bo, _, _ = run_both(d2, p2, b2, 2)
    for v in range(8):
        assert np.abs(pg[v] - po[v]).max() <= 1e-11 * np.abs(po[v]).max(), v
    assert np.abs(bg - bo).max() <= 1e-11 * np.abs(bo).max()


def test_ragged_block_and_fixed_dt():
    """Sizes that are not multiples of any tile or warp, and a caller-fixed dt."""
    geo, d, prim, bf = torus_case(21, 13, 6, seed=5)
    pg, bg, po, bo, dts, _ = run_both(d, prim, bf, 2, dt=0.01)
    assert all(a == 0.01 and b == 0.01 for a, b in dts)
    assert_parity(*field_errors(d, pg, bg, po, bo), 1e-11)


def test_div_b_stays_at_roundoff_on_gpu():
    geo, d, prim, bf = torus_case(32, 16, 8, seed=4)
    g = gpu_grid(d)
    g.set_state(prim, bf)
    for _ in range(5):
        g.step()
    _, b = g.get_state()
    g.close()
    s = NG
    n1, n2, n3 = d.n1, d.n2, d.n3
    div = ((b[0][s:s + n3, s:s + n2, s + 1:s + n1 + 1] - b[0][s:s + n3, s:s + n2, s:s + n1]) / d.dx1
           + (b[1][s:s + n3, s + 1:s + n2 + 1, s:s + n1] - b[1][s:s + n3, s:s + n2, s:s + n1]) / d.dx2
           + (b[2][s + 1:s + n3 + 1, s:s + n2, s:s + n1] - b[2][s:s + n3, s:s + n2, s:s + n1]) / d.dx3)
    assert np.abs(div).max() < 1e-13 * np.abs(b).max() / min(d.dx1, d.dx2, d.dx3)


def test_step_parity_torus_256x128x64_full_size():
    """The benchmark's block and launch configuration, one step, every cell."""
    geo, d, prim, bf = torus_case(256, 128, 64, seed=10192)
    pg, bg, po, bo, dts, _ = run_both(d, prim, bf, 1)
    assert abs(dts[0][0] - dts[0][1]) <= 1e-13 * dts[0][1]
    assert_parity(*field_errors(d, pg, bg, po, bo), 1e-12)


def test_llf_and_minmod_options_parity():
    geo, d, prim, bf = torus_case(32, 16, 8, seed=9, recon=O.RECON_MINMOD, riemann=O.FLUX_LLF)
    pg, bg, po, bo, _, _ = run_both(d, prim, bf, 2)
    assert_parity(*field_errors(d, pg, bg, po, bo), 1e-11)


def test_bondi_and_shock_tube_parity():
    """The FP64 path against the oracle on the two validation set-ups of the oracle's pins: Michel
    accretion (Kerr-Schild a = 0, theta band, zero-gradient boundaries) and the relativistic blast
    wave (flat space, periodic transverse directions), ten steps each at the 10-step bar."""
    geo = W.BlockGeometry(64, 4, 4, math.log(1.8), math.log(20.0), math.pi / 2 - 0.2, math.pi / 2 + 0.2, 0.0, 0.2)
    prim, bf = W.bondi_block(geo)
    d = O.make_desc(64, 4, 4, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3, metric=O.METRIC_KS,
                    a=0.0, gam=4.0 / 3.0, cour=0.8, bc=(0, 0, 0, 0, 1, 1), floors=0)
    pg, bg, po, bo, dts, _ = run_both(d, prim, bf, 10)
    errs, _ = field_errors(d, pg, bg, po, bo)
    for k in ("rho", "u", "utilde"):
        assert errs[k] <= 1e-9, (k, errs)
    assert not np.any(bg) and not np.any(bo)  # no field: it stays zero

    n1, gam = 200, 5.0 / 3.0
    d = O.make_desc(n1, 4, 4, 0.0, 0.0, 0.0, 1.0 / n1, 1.0, 1.0, metric=O.METRIC_MINKOWSKI, gam=gam, cour=0.5,
                    recon=O.RECON_PPM, riemann=O.FLUX_HLL, bc=(0, 0, 1, 1, 1, 1), floors=0)
    prim = np.zeros((8, 10, 10, n1 + 2 * NG))
    x = (np.arange(-NG, n1 + NG) + 0.5) / n1
    prim[0][...] = np.where(x < 0.5, 10.0, 1.0)[None, None, :]
    prim[1][...] = (np.where(x < 0.5, 13.33, 1e-6) / (gam - 1.0))[None, None, :]
    pg, bg, po, bo, dts, _ = run_both(d, prim, np.zeros((3,) + prim.shape[1:]), 10)
    errs, _ = field_errors(d, pg, bg, po, bo)
    for k in ("rho", "u", "utilde"):
        assert errs[k] <= 1e-9, (k, errs)


@pytest.mark.parametrize("nsteps,bar", [(1, 1e-12), (10, 1e-9)])
def test_upwinded_emf_parity_torus(nsteps, bar):
    """Upwinded EMFs (Gardiner & Stone 2005) on the 64x32x16 torus: the FP64 bars."""
    geo, d, prim, bf = torus_case(64, 32, 16, seed=1912)
    d.emf = O.EMF_UPWIND
    pg, bg, po, bo, dts, _ = run_both(d, prim, bf, nsteps)
    assert_parity(*field_errors(d, pg, bg, po, bo), bar)


def test_field_loop_parity_and_upwinding_gain():
    """Field-loop advection through the CUDA path with both EMF forms: the oracle's result after 40
    steps (1e-9), and over a whole crossing at 128^2 the upwinded loop returns closer to its start."""
    from paper_1912_10192_gb300 import hamr
    for emf in (O.EMF_AVERAGE, O.EMF_UPWIND):
        prim, bf, dx1, dx2 = W.field_loop_block(32, 32, v=(0.4, 0.4))
        d = O.make_desc(32, 32, 4, -0.5, -0.5, 0.0, dx1, dx2, 1.0, metric=O.METRIC_MINKOWSKI, gam=5.0 / 3.0,
                        cour=0.5, bc=(1,) * 6, floors=0, emf=emf)
        pg, bg, po, bo, _, _ = run_both(d, prim, bf, 40)
        fg, fo = face_interior(bg, d)[:2], face_interior(bo, d)[:2]
        e = sum(np.abs(x - y).sum() for x, y in zip(fg, fo)) / sum(np.abs(y).sum() for y in fo)
        assert e <= 1e-9, (emf, e)
    errs = {}
    n = 128
    for emf in (hamr.EMF_AVERAGE, hamr.EMF_UPWIND):
        prim, bf, dx1, dx2 = W.field_loop_block(n, n, v=(0.4, 0.4))
        b = hamr.block(n, n, 4, -0.5, -0.5, 0.0, dx1, dx2, 1.0, (1,) * 6)
        g = hamr.Grid([b], metric=hamr.METRIC_MINKOWSKI, gam=5.0 / 3.0, cour=0.5, floors=0, emf=emf)
        g.set_state(torch.from_numpy(prim).cuda(), torch.from_numpy(bf).cuda())
        t, T = 0.0, 1.0 / 0.4
        while t < T - 1e-12:
            st = g.step(stats=True)
            t += st["dt_used"]
            if T - t < st["dt_next"]:
                g.step(T - t)
                t = T
        _, bo = g.get_state()
        g.close()
        f = [(bo[0][NG + 1, NG:NG + n, NG:NG + n + 1], bf[0][NG + 1, NG:NG + n, NG:NG + n + 1]),
             (bo[1][NG + 1, NG:NG + n + 1, NG:NG + n], bf[1][NG + 1, NG:NG + n + 1, NG:NG + n])]
        errs[emf] = sum(np.abs(x - x0).sum() for x, x0 in f) / sum(np.abs(x0).sum() for _, x0 in f)
    print("field loop, 128^2, one crossing, L1 of the face field:", errs)
    assert errs[hamr.EMF_UPWIND] < 0.6 * errs[hamr.EMF_AVERAGE]
