"""Grid-level pins of the oracle's step (Sec. 2.1, 2.5): constrained transport,
conservation, free streaming, convergence order, advection and equilibrium."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

NG = O.NG
GAM = 13.0 / 9.0


def torus_desc(n1, n2, n3, recon=O.RECON_PPM):
    geo = W.torus_geometry(n1, n2, n3)
    d = O.make_desc(n1, n2, n3, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3,
                    metric=O.METRIC_KS, a=0.9375, gam=GAM, cour=0.8, recon=recon,
                    bc=(O.BC_OUTFLOW_NOINFLOW, O.BC_OUTFLOW_NOINFLOW, O.BC_POLAR, O.BC_POLAR,
                        O.BC_PERIODIC, O.BC_PERIODIC))
    return geo, d


def flat_desc(n1, n2, n3, L=(1.0, 1.0, 1.0), gam=GAM, recon=O.RECON_PPM, cour=0.8):
    return O.make_desc(n1, n2, n3, 0.0, 0.0, 0.0, L[0] / n1, L[1] / n2, L[2] / n3,
                       metric=O.METRIC_MINKOWSKI, gam=gam, cour=cour, recon=recon,
                       bc=(O.BC_PERIODIC,) * 6, floors=0)


def interior(a, d):
    return a[..., NG:NG + d.n3, NG:NG + d.n2, NG:NG + d.n1]


@pytest.mark.parametrize("emf", [O.EMF_AVERAGE, O.EMF_UPWIND])
def test_ct_keeps_div_b_at_roundoff_on_torus(emf):
    geo, d = torus_desc(32, 16, 8)
    d.emf = emf
    prim, bf = W.torus_block(geo, seed=1912)
    g = O.Grid(d)
    g.set(prim, bf)
    scale = np.abs(bf).max() / min(d.dx1, d.dx2, d.dx3)
    assert np.abs(g.divb()).max() < 1e-14 * scale
    for _ in range(4):
        g.step()
    assert np.abs(g.divb()).max() < 1e-13 * scale


def _flat_random_state(d, seed, amp=0.1):
    rng = np.random.default_rng(seed)
    shp = (d.n3 + 2 * NG, d.n2 + 2 * NG, d.n1 + 2 * NG)
    prim = np.zeros((8,) + shp)
    bf = np.zeros((3,) + shp)
    x = (np.arange(d.n1) + 0.5) * d.dx1
    y = (np.arange(d.n2) + 0.5) * d.dx2
    z = (np.arange(d.n3) + 0.5) * d.dx3
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    tp = 2 * math.pi
    s = (slice(NG, NG + d.n3), slice(NG, NG + d.n2), slice(NG, NG + d.n1))
    prim[0][s] = 1.0 + amp * np.sin(tp * X + 1) * np.cos(tp * Y)
    prim[1][s] = 1.0 + amp * np.cos(tp * Z + 2 * tp * X)
    prim[2][s] = 0.3 + amp * np.sin(tp * Y)
    prim[3][s] = -0.2 + amp * np.sin(tp * (X + Z))
    prim[4][s] = 0.1 + amp * np.cos(tp * X)
    # face B as the discrete curl of a periodic edge vector potential A = (A1(y,z), 0, A3(x,y))
    xf = np.arange(d.n1) * d.dx1
    yf = np.arange(d.n2) * d.dx2
    zf = np.arange(d.n3) * d.dx3
    YF, XF = np.meshgrid(yf, xf, indexing="ij")
    a3 = 0.05 * np.sin(tp * XF) * np.sin(tp * YF) / tp          # edges (i-1/2, j-1/2), [j, i]
    ZF, YF2 = np.meshgrid(zf, yf, indexing="ij")
    a1 = 0.05 * np.cos(tp * YF2 + tp * ZF) / tp                # edges (j-1/2, k-1/2), [k, j]
    b1 = (np.roll(a3, -1, axis=0) - a3) / d.dx2                 # [j, i]
    b2 = ((np.roll(a1, -1, axis=0) - a1) / d.dx3)[:, :, None] - ((np.roll(a3, -1, axis=1) - a3) / d.dx1)[None]
    b3 = -(np.roll(a1, -1, axis=1) - a1) / d.dx2                # [k, j]
    bf[0][s] = np.broadcast_to(b1[None], (d.n3, d.n2, d.n1))
    bf[1][s] = b2
    bf[2][s] = np.broadcast_to(b3[:, :, None], (d.n3, d.n2, d.n1))
    return prim, bf


def _total_U(d, prim):
    p = interior(prim, d).reshape(8, -1).T
    n = p.shape[0]
    U = O.p2u_many(d, p, np.zeros(n), np.zeros(n))
    return U.sum(axis=0)


def test_flat_periodic_box_conserves_and_keeps_div_b():
    d = flat_desc(16, 12, 8)
    prim, bf = _flat_random_state(d, 1)
    g = O.Grid(d)
    g.set(prim, bf)
    assert np.abs(g.divb()).max() < 1e-12
    p0, _ = g.get()
    U0 = _total_U(d, p0)
    for _ in range(5):
        g.step()
    p1, _ = g.get()
    U1 = _total_U(d, p1)
    assert g.stats()[1:3] == [0, 0]
    # mass, energy, momenta: conserved to round-off (the inversion adds ~1e-14 per cell)
    for m in range(5):
        assert abs(U1[m] - U0[m]) < 1e-12 * np.abs(U0[:5]).max()
    assert np.abs(g.divb()).max() < 1e-12


def test_free_streaming_uniform_state():
    d = flat_desc(8, 8, 8)
    shp = (d.n3 + 2 * NG, d.n2 + 2 * NG, d.n1 + 2 * NG)
    prim = np.zeros((8,) + shp)
    bf = np.zeros((3,) + shp)
    vals = [1.3, 0.7, 0.4, -0.3, 0.2]
    for v, x in enumerate(vals):
        prim[v][...] = x
    bf[0][...], bf[1][...], bf[2][...] = 0.2, -0.1, 0.3
    g = O.Grid(d)
    g.set(prim, bf)
    for _ in range(3):
        g.step()
    p, b = g.get()
    for v, x in enumerate(vals):
        assert np.abs(interior(p[v], d) - x).max() < 1e-13 * max(1, abs(x))
    assert np.abs(interior(b[0], d) - 0.2).max() < 1e-15


def _sound_wave_error(n, recon):
    gam = 5.0 / 3.0
    d = flat_desc(n, 1, 1, L=(1.0, 1.0 / n, 1.0 / n), gam=gam, recon=recon, cour=0.5)
    rho0, u0, A = 1.0, 1.0, 1e-5
    p0 = (gam - 1) * u0
    w0 = rho0 + u0 + p0
    cs = math.sqrt(gam * p0 / w0)
    x = (np.arange(n) + 0.5) / n
    shp = (d.n3 + 2 * NG, d.n2 + 2 * NG, d.n1 + 2 * NG)
    prim = np.zeros((8,) + shp)
    bf = np.zeros((3,) + shp)
    # cell averages of the right-going eigenmode: drho = A rho0 cos, de = (w0/rho0) drho, v = cs drho/rho0
    ca = (np.sin(2 * math.pi * (x + 0.5 / n)) - np.sin(2 * math.pi * (x - 0.5 / n))) * n / (2 * math.pi)
    drho = A * rho0 * ca
    prim[0][NG, NG, NG:NG + n] = rho0 + drho
    prim[1][NG, NG, NG:NG + n] = u0 + (w0 / rho0 - 1.0) * drho
    prim[2][NG, NG, NG:NG + n] = cs * drho / rho0
    init = prim[0][NG, NG, NG:NG + n].copy()
    g = O.Grid(d)
    g.set(prim, bf)
    T = 1.0 / cs
    t = 0.0
    while t < T - 1e-14:
        dt = min(g.dt(), T - t)
        g.step(dt)
        t += dt
    p, _ = g.get()
    return np.abs(p[0][NG, NG, NG:NG + n] - init).mean()


@pytest.mark.parametrize("recon", [O.RECON_PPM, O.RECON_MC])
def test_linear_sound_wave_converges_at_second_order(recon):
    """Sec. 6.1: linear waves converge at 2nd order (one period, flat space)."""
    e = [_sound_wave_error(n, recon) for n in (32, 64, 128)]
    rates = [math.log2(e[0] / e[1]), math.log2(e[1] / e[2])]
    assert min(rates) > 1.7, (e, rates)


def test_weak_field_is_advected_downstream():
    """A passive transverse field in a uniform flow moves with the flow: checks the sign of
    the induction flux F^j(B^i) = b^i u^j - b^j u^i together with the CT update."""
    n = 64
    d = flat_desc(n, 1, 1, L=(1.0, 1.0 / n, 1.0 / n), recon=O.RECON_PPM, cour=0.5)
    shp = (d.n3 + 2 * NG, d.n2 + 2 * NG, d.n1 + 2 * NG)
    prim = np.zeros((8,) + shp)
    bf = np.zeros((3,) + shp)
    v = 0.5
    Wl = 1 / math.sqrt(1 - v * v)
    prim[0][...] = 1.0
    prim[1][...] = 1.0
    prim[2][...] = Wl * v
    x = (np.arange(n) + 0.5) / n
    By = 1e-4 * np.exp(-((x - 0.3) / 0.08) ** 2)
    bf[1][NG, NG:NG + 2, NG:NG + n] = By  # x2-faces (uniform in y)
    g = O.Grid(d)
    g.set(prim, bf)
    T = 0.4 / v
    t = 0.0
    while t < T - 1e-14:
        dt = min(g.dt(), T - t)
        g.step(dt)
        t += dt
    _, b = g.get()
    prof = b[1][NG, NG, NG:NG + n]
    centre = (prof * x).sum() / prof.sum()
    assert abs(centre - 0.7) < 0.01, centre


def test_torus_hydrostatic_balance_converges():
    """The FM torus is an exact equilibrium: div F - Q of the exact state, with the
    oracle's fluxes, sources and metric, vanishes at 2nd order in the spacing."""
    a, gam = 0.9375, GAM
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=a, gam=gam)
    ell = W.fm_ell(a, 12.0)
    lnh_in = W._fm_lnh(a, 6.0, math.pi / 2, ell)
    kappa = 1e-3

    def prim_at(x1, x2):
        r, th = math.exp(x1), x2
        h = math.exp(W._fm_lnh(a, r, th, ell) - lnh_in)
        rho = ((h - 1) * (gam - 1) / (kappa * gam)) ** (1 / (gam - 1))
        u = kappa * rho ** gam / (gam - 1)
        ut, up = W._fm_velocity_bl(a, np.array(r), np.array(th), ell)
        _, gtt, gt1, _ = W._ks_internal(a, np.array(r), np.array(th))
        al = 1 / math.sqrt(-gtt)
        return np.array([rho, u, float(al * ut * al * gt1), 0.0, float(up), 0, 0, 0])

    for (x1, x2) in [(math.log(12.0), 1.5), (math.log(9.0), 1.3)]:
        res = []
        for h in (1e-2, 5e-3):
            div = np.zeros(9)
            for dr, (o1, o2) in ((1, (h, 0)), (2, (0, h))):
                Fp = O.p2uf(d, prim_at(x1 + o1 / 2, x2 + o2 / 2), x1 + o1 / 2, x2 + o2 / 2, dr)
                Fm = O.p2uf(d, prim_at(x1 - o1 / 2, x2 - o2 / 2), x1 - o1 / 2, x2 - o2 / 2, dr)
                div += (Fp - Fm) / h
            Q = O.source(d, prim_at(x1, x2), x1, x2)
            res.append(np.abs(div[1:5] - Q[1:5]).max() / np.abs(Q[1:5]).max())
        assert res[0] < 1e-3 and 3.5 < res[0] / res[1] < 4.5, res


def test_torus_step_runs_and_uses_documented_fallbacks():
    geo, d = torus_desc(32, 16, 8)
    prim, bf = W.torus_block(geo, seed=1912)
    g = O.Grid(d)
    g.set(prim, bf)
    dt0 = g.dt()
    assert 0.0 < dt0 < 1.0
    for _ in range(2):
        g.step()
    p, b = g.get()
    assert np.isfinite(p).all() and np.isfinite(b).all()
    st = g.stats()
    ncell = 2 * d.n1 * d.n2 * d.n3
    assert st[0] > 0.85 * ncell and st[2] < 0.02 * ncell


def _bondi_run(n1, recon, T=5.0):
    from paper_1912_10192_gb300 import workloads as W
    geo = W.BlockGeometry(n1, 4, 4, math.log(1.8), math.log(20.0), math.pi / 2 - 0.2, math.pi / 2 + 0.2, 0.0, 0.2)
    prim, bf = W.bondi_block(geo)
    d = O.make_desc(n1, 4, 4, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3, metric=O.METRIC_KS, a=0.0,
                    gam=4.0 / 3.0, cour=0.8, recon=recon, bc=(0, 0, 0, 0, 1, 1), floors=0)
    g = O.Grid(d)
    g.set(prim, bf)
    t = 0.0
    while t < T:
        t += g.step()
    p, _ = g.get()
    r = np.exp(geo.x1min + (np.arange(n1) + 0.5) * geo.dx1)
    e = (p[0][NG + 1, NG + 2, NG:NG + n1] - prim[0][NG, NG, NG:NG + n1]) / prim[0][NG, NG, NG:NG + n1]
    return r, e, g.stats()


def test_bondi_inflow_stays_stationary():
    """Michel's spherical accretion onto a Schwarzschild hole (rc = 8, Gamma = 4/3), r 1.8..20 in a
    theta band with zero-gradient boundaries, t = 5: the exact solution is a steady state of the
    scheme up to truncation. With MC slopes the density error over r 2.5..16 is < 1e-4 and falls
    with resolution; with PPM the subsonic part (r > 9) stays within 1e-5, while the supersonic part
    carries an odd-even pattern of first-order amplitude (the centred PPM interface values do not see
    that mode, and fully upwind fluxes do not damp it), which this test bounds at 2e-2 and halves
    with the cell size."""
    r64, e64, st = _bondi_run(64, O.RECON_MC)
    r128, e128, _ = _bondi_run(128, O.RECON_MC)
    assert st[1] == 0 and st[2] == 0  # every inversion by the energy equation
    s64, s128 = (r64 > 2.5) & (r64 < 16), (r128 > 2.5) & (r128 < 16)
    m64, m128 = np.abs(e64[s64]).mean(), np.abs(e128[s128]).mean()
    assert m64 < 1e-4 and m128 < 0.75 * m64, (m64, m128)
    r64, p64, _ = _bondi_run(64, O.RECON_PPM)
    r128, p128, _ = _bondi_run(128, O.RECON_PPM)
    assert np.abs(p64[(r64 > 9) & (r64 < 16)]).mean() < 1e-5
    a64 = np.abs(p64[(r64 > 2.5) & (r64 < 7)]).mean()
    a128 = np.abs(p128[(r128 > 2.5) & (r128 < 7)]).mean()
    assert a64 < 2e-2 and 1.6 < a64 / a128 < 2.6, (a64, a128)


def _shock_tube(n1, recon, T=0.4):
    """Marti & Mueller (1999) problem 1 along x1 of a flat-space block: rho 10, p 13.33 | rho 1, p 1e-6,
    Gamma 5/3, at rest, interface at x = 0.5; L1 errors of rho and v against the exact solution."""
    import srhd_exact as X
    gam = 5.0 / 3.0
    d = O.make_desc(n1, 4, 4, 0.0, 0.0, 0.0, 1.0 / n1, 1.0, 1.0, metric=O.METRIC_MINKOWSKI, gam=gam, cour=0.5,
                    recon=recon, riemann=O.FLUX_HLL, bc=(0, 0, 1, 1, 1, 1), floors=0)
    prim = np.zeros((8, 10, 10, n1 + 2 * NG))
    x = (np.arange(-NG, n1 + NG) + 0.5) / n1
    left = x < 0.5
    prim[0][...] = np.where(left, 10.0, 1.0)[None, None, :]
    prim[1][...] = (np.where(left, 13.33, 1e-6) / (gam - 1.0))[None, None, :]
    g = O.Grid(d)
    g.set(prim, np.zeros((3,) + prim.shape[1:]))
    t = 0.0
    while t < T - 1e-13:
        t += g.step(min(g.dt(), T - t))
    p, _ = g.get()
    L, R = X.State(10.0, 13.33, 0.0, gam), X.State(1.0, 1e-6, 0.0, gam)
    xc = (np.arange(n1) + 0.5) / n1
    ex = np.array([X.sample(L, R, (xx - 0.5) / T) for xx in xc])
    rho = p[0][NG + 1, NG + 1, NG:NG + n1]
    ut = p[2][NG + 1, NG + 1, NG:NG + n1]
    v = ut / np.sqrt(1.0 + ut * ut)
    return np.abs(rho - ex[:, 0]).mean(), np.abs(v - ex[:, 2]).mean()


def test_exact_riemann_solver_reference():
    """The exact solver itself: Newtonian limit against Toro's Sod values (pressures scaled by 1e-5),
    Marti & Mueller's problem 1 star state, and Rankine-Hugoniot across its shock."""
    import srhd_exact as X
    s = 1e-5
    ps, vs, SL, SR, _, vsr = X.solve(X.State(1.0, s, 0.0, 1.4), X.State(0.125, 0.1 * s, 0.0, 1.4))
    assert abs(ps / s - 0.30313) < 2e-5 and abs(vs / math.sqrt(s) - 0.92745) < 5e-5
    assert abs(SL.rho - 0.42632) < 2e-5 and abs(SR.rho - 0.26557) < 2e-5
    L, R = X.State(10.0, 13.33, 0.0, 5.0 / 3.0), X.State(1.0, 1e-6, 0.0, 5.0 / 3.0)
    ps, vs, SL, SR, _, vsr = X.solve(L, R)
    assert abs(ps - 1.448) < 1e-3 and abs(vs - 0.714) < 1e-3 and abs(SR.rho - 5.07) < 1e-2 and abs(vsr - 0.828) < 1e-3

    def uf(st):
        W, h = st.W, st.h
        return ((st.rho * W, st.rho * h * W * W * st.v, st.rho * h * W * W - st.p),
                (st.rho * W * st.v, st.rho * h * W * W * st.v * st.v + st.p, st.rho * h * W * W * st.v))
    (ua, fa), (ub, fb) = uf(R), uf(SR)
    for q in range(3):
        assert abs((fb[q] - vsr * ub[q]) - (fa[q] - vsr * ua[q])) < 1e-12 * max(1.0, abs(fa[q]))


def test_relativistic_shock_tube_converges_to_the_exact_solution():
    """Shock capturing (Sec. 2.1: PPM or MINMOD edge values, HLL fluxes) on the relativistic blast of
    Marti & Mueller problem 1 at t = 0.4: first-order convergence of the L1 errors toward the exact
    solution (shocks and the contact are smeared over a fixed number of cells), PPM sharper than
    MINMOD."""
    e100 = _shock_tube(100, O.RECON_PPM)
    e200 = _shock_tube(200, O.RECON_PPM)
    m200 = _shock_tube(200, O.RECON_MINMOD)
    assert e200[0] < 0.07 and e200[1] < 0.01, e200
    assert e200[0] < 0.65 * e100[0] and e200[1] < 0.65 * e100[1], (e100, e200)
    assert m200[0] > 1.5 * e200[0], (m200, e200)


def _field_loop(n, emf, v=(0.4, 0.4)):
    prim, bf, dx1, dx2 = W.field_loop_block(n, n, v=v)
    d = O.make_desc(n, n, 4, -0.5, -0.5, 0.0, dx1, dx2, 1.0, metric=O.METRIC_MINKOWSKI, gam=5.0 / 3.0, cour=0.5,
                    bc=(1, 1, 1, 1, 1, 1), floors=0, emf=emf)
    g = O.Grid(d)
    g.set(prim, bf)
    T = 1.0 / v[0]  # one crossing along x1 and x2: the loop is back where it started
    t = 0.0
    while t < T - 1e-13:
        t += g.step(min(g.dt(), T - t))
    _, b = g.get()
    f = [(b[0][NG + 1, NG:NG + n, NG:NG + n + 1], bf[0][NG + 1, NG:NG + n, NG:NG + n + 1]),
         (b[1][NG + 1, NG:NG + n + 1, NG:NG + n], bf[1][NG + 1, NG:NG + n + 1, NG:NG + n])]
    err = sum(np.abs(x - x0).sum() for x, x0 in f) / sum(np.abs(x0).sum() for _, x0 in f)
    me = sum((x * x).sum() for x, _ in f) / sum((x0 * x0).sum() for _, x0 in f)
    scale = np.abs(bf).max() / min(dx1, dx2)
    return err, me, np.abs(g.divb()).max() / scale, np.abs(b[2]).max()


def test_upwinded_emfs_reduce_to_the_average_for_uniform_emf():
    """A uniform magnetised flow: every face and cell EMF is equal, the Gardiner-Stone corrections
    vanish, and both EMF forms give the same step to round-off."""
    d = flat_desc(8, 8, 8)
    shp = (14, 14, 14)
    prim = np.zeros((8,) + shp)
    bf = np.zeros((3,) + shp)
    prim[0][...], prim[1][...], prim[2][...], prim[3][...], prim[4][...] = 1.0, 0.5, 0.3, -0.2, 0.1
    bf[0][...], bf[1][...], bf[2][...] = 0.2, -0.1, 0.05
    res = []
    for emf in (O.EMF_AVERAGE, O.EMF_UPWIND):
        d.emf = emf
        g = O.Grid(d)
        g.set(prim, bf)
        g.step(0.01)
        res.append(g.get())
    assert np.abs(res[0][0] - res[1][0]).max() < 1e-15 and np.abs(res[0][1] - res[1][1]).max() < 1e-15


def test_field_loop_is_cleaner_with_upwinded_emfs():
    """Gardiner & Stone (2005) field-loop advection in flat space (weak loop, beta >> 1, diagonal
    flow, one crossing of the periodic box): with upwinded EMFs the loop returns closer to its start
    (L1 of the face field), with div B at round-off and no field along x3 in both forms."""
    e_avg, me_avg, div_avg, b3_avg = _field_loop(32, O.EMF_AVERAGE)
    e_up, me_up, div_up, b3_up = _field_loop(32, O.EMF_UPWIND)
    assert e_up < 0.6 * e_avg, (e_up, e_avg)
    assert me_up > 0.8 and me_avg > 0.8, (me_up, me_avg)
    assert div_up < 1e-13 and div_avg < 1e-13
    assert b3_up == 0.0 and b3_avg == 0.0
