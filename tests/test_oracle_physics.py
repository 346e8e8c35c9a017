"""Pins of the oracle's point-wise physics (Sec. 2.1, 2.3-2.6) against
textbook special-relativistic MHD, invariants and consistency properties."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

GAM = 13.0 / 9.0


def _ks(a=0.9375):
    return O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=a, gam=GAM)


def _flat(gam=GAM):
    return O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_MINKOWSKI, gam=gam)


def test_normalisation_on_random_states():
    d = _ks()
    prim, x1, x2 = W.random_states(300, seed=11)
    for p, a1, a2 in zip(prim, x1, x2):
        ucon, ucov, bcon, bcov, bsq = O.state(d, p, a1, a2)
        assert abs(ucon @ ucov + 1.0) < 1e-12 * max(1.0, ucon[0] * abs(ucov[0]))
        assert abs(bcon @ ucov) < 1e-12 * (np.abs(bcon) @ np.abs(ucov) + 1e-300)
        # B^i = F*^{it} = b^i u^t - b^t u^i (Sec. 2.3)
        for i in range(1, 4):
            assert abs(bcon[i] * ucon[0] - bcon[0] * ucon[i] - p[4 + i]) < 1e-11 * (abs(p[4 + i]) + 1e-300) \
                + 1e-13 * np.abs(bcon).max() * np.abs(ucon).max()


def _srmhd_textbook(p, gam):
    """Flat-space SRMHD in the lab frame: v^i, Lorentz factor W, B^i (B = F*^{it})."""
    rho, u = p[0], p[1]
    ut = np.array(p[2:5])
    Wl = math.sqrt(1.0 + ut @ ut)
    v = ut / Wl
    B = np.array(p[5:8])
    pg = (gam - 1.0) * u
    h = rho + u + pg
    b0 = Wl * (B @ v)
    bvec = B / Wl + b0 * v
    b2 = (B @ B) / Wl ** 2 + (B @ v) ** 2
    T00 = (h + b2) * Wl ** 2 - (pg + 0.5 * b2) - b0 ** 2
    T0i = (h + b2) * Wl ** 2 * v - b0 * bvec
    Tij = (h + b2) * Wl ** 2 * np.outer(v, v) + (pg + 0.5 * b2) * np.eye(3) - np.outer(bvec, bvec)
    kappa = pg / rho ** gam
    return dict(D=rho * Wl, v=v, W=Wl, B=B, T00=T00, T0i=T0i, Tij=Tij, kappa=kappa, rho=rho)


def test_flat_conserved_and_fluxes_match_textbook_srmhd():
    """U and F^x of the covariant oracle reduce to the textbook SRMHD forms, including
    the b^2 u u term of T and the induction flux v^j B^i - v^i B^j."""
    d = _flat()
    rng = np.random.default_rng(3)
    for _ in range(50):
        p = np.concatenate([[rng.uniform(0.1, 2), rng.uniform(0.01, 3)], rng.normal(0, 1.5, 3),
                            rng.normal(0, 1.0, 3)])
        t = _srmhd_textbook(p, GAM)
        U = O.p2uf(d, p, 0.0, 0.0, 0)
        # lowering t flips sign: T^t_t = -T^{00}, T^t_i = T^{0i}
        ref_U = [t["D"], -t["T00"] + t["D"], *t["T0i"], t["kappa"] * t["D"], *t["B"]]
        assert np.allclose(U, ref_U, rtol=1e-12, atol=1e-12 * np.abs(ref_U).max())
        for j in range(3):
            F = O.p2uf(d, p, 0.0, 0.0, j + 1)
            vj = t["v"][j]
            mass = t["D"] * vj
            ref_F = [mass, -t["T0i"][j] + mass, *t["Tij"][j], t["kappa"] * mass,
                     *[t["B"][i] * vj - t["B"][j] * t["v"][i] for i in range(3)]]
            assert np.allclose(F, ref_F, rtol=1e-12, atol=1e-12 * np.abs(ref_F).max())


def test_sound_speed_reduces_to_relativistic_velocity_addition():
    """B = 0 flow along x in flat space: v+- = (v +- cs)/(1 +- v cs)."""
    d = _flat()
    for v in [0.0, 0.3, -0.7, 0.95]:
        rho, u = 1.0, 0.7
        Wl = 1 / math.sqrt(1 - v * v)
        p = np.array([rho, u, Wl * v, 0, 0, 0, 0, 0])
        pg = (GAM - 1) * u
        cs = math.sqrt(GAM * pg / (rho + u + pg))
        vp, vm = O.vchar(d, p, 0, 0, 1)
        assert abs(vp - (v + cs) / (1 + v * cs)) < 1e-14
        assert abs(vm - (v - cs) / (1 - v * cs)) < 1e-14
        # transverse direction: +-cs/W for a flow along x (speed of a wave along y)
        vp2, vm2 = O.vchar(d, p, 0, 0, 2)
        assert abs(vp2 + vm2) < 1e-14 and vp2 > 0


def test_static_magnetised_fast_speed():
    """Static gas: the speed is the fluid-frame magnetosonic speed sqrt(vA^2 + cs^2 (1 - vA^2))."""
    d = _flat()
    rho, u, Bx = 1.0, 0.5, 0.8
    p = np.array([rho, u, 0, 0, 0, Bx, 0, 0])
    pg = (GAM - 1) * u
    w = rho + u + pg
    cs2 = GAM * pg / w
    va2 = Bx * Bx / (Bx * Bx + w)
    c = math.sqrt(va2 + cs2 * (1 - va2))
    for dr in (1, 2, 3):
        vp, vm = O.vchar(d, p, 0, 0, dr)
        assert abs(vp - c) < 1e-14 and abs(vm + c) < 1e-14


@pytest.mark.parametrize("riemann", [O.FLUX_HLL, O.FLUX_LLF])
def test_riemann_consistency(riemann):
    """F(U, U) = F(U) on curved-space random states (sqrt(-g) at the face)."""
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=GAM, riemann=riemann)
    prim, x1, x2 = W.random_states(100, seed=12)
    for p, a1, a2 in zip(prim, x1, x2):
        for dr in (1, 2, 3):
            F = O.face_flux(d, p, p, a1, a2, dr)
            ref = O.p2uf(d, p, a1, a2, dr)
            keep = [0, 1, 2, 3, 4, 5] + [5 + i for i in (1, 2, 3) if i != dr]
            assert np.allclose(F, ref[keep], rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_hll_upwinds_supersonic_flow():
    d = _flat()
    pl = np.array([1.0, 0.1, 5.0, 0.3, 0.0, 0.1, 0.2, 0.0])
    pr = np.array([0.8, 0.12, 4.5, 0.2, 0.1, 0.1, 0.25, 0.05])
    F = O.face_flux(d, pl, pr, 0, 0, 1)
    FL = O.p2uf(d, pl, 0, 0, 1)
    assert O.vchar(d, pr, 0, 0, 1)[1] > 0 and O.vchar(d, pl, 0, 0, 1)[1] > 0
    assert np.allclose(F, FL[[0, 1, 2, 3, 4, 5, 7, 8]], rtol=1e-14, atol=1e-15)


def test_hll_flux_is_hll_of_two_states():
    """Where both states move subsonically the HLL flux lies between one-sided fluxes
    in the sense of the integral form: F = F_L - cmin... checked by the HLL identity
    (cmax + cmin) F = cmin F_R + cmax F_L - cmax cmin (U_R - U_L)."""
    d = _flat()
    pl = np.array([1.0, 1.0, 0.1, 0.0, 0.0, 0.3, 0.2, 0.1])
    pr = np.array([0.125, 0.1, 0.0, 0.0, 0.0, 0.3, -0.2, 0.0])
    vpl, vml = O.vchar(d, pl, 0, 0, 1)
    vpr, vmr = O.vchar(d, pr, 0, 0, 1)
    cmax = max(0, vpl, vpr)
    cmin = max(0, -vml, -vmr)
    keep = [0, 1, 2, 3, 4, 5, 7, 8]
    FL, FR = O.p2uf(d, pl, 0, 0, 1)[keep], O.p2uf(d, pr, 0, 0, 1)[keep]
    UL, UR = O.p2uf(d, pl, 0, 0, 0)[keep], O.p2uf(d, pr, 0, 0, 0)[keep]
    F = O.face_flux(d, pl, pr, 0, 0, 1)
    assert np.allclose((cmax + cmin) * F, cmin * FR + cmax * FL - cmax * cmin * (UR - UL), atol=1e-14)


def test_ppm_exact_for_linear_and_cubic_averages():
    x = np.linspace(1.0, 2.0, 21)
    # cell averages of f = x^3 + 2x over [x_c, x_c+1]
    F = lambda y: y ** 4 / 4 + y ** 2
    q = (F(x[1:]) - F(x[:-1])) / (x[1:] - x[:-1])
    al, ar = O.recon_line(O.RECON_PPM, q)
    f = lambda y: y ** 3 + 2 * y
    n = len(q)
    for c in range(2, n - 2):
        assert abs(al[c] - f(x[c])) < 1e-12 and abs(ar[c] - f(x[c + 1])) < 1e-12
    ql = 3.0 * np.arange(12) - 4.0
    for recon in (O.RECON_PPM, O.RECON_MC, O.RECON_MINMOD):
        al, ar = O.recon_line(recon, ql)
        lo = 2 if recon == O.RECON_PPM else 1
        for c in range(lo, 12 - lo):
            assert abs(al[c] - (ql[c] - 1.5)) < 1e-13 and abs(ar[c] - (ql[c] + 1.5)) < 1e-13


def test_ppm_monotone_and_flat_at_extrema():
    rng = np.random.default_rng(5)
    for _ in range(200):
        q = rng.normal(size=16)
        al, ar = O.recon_line(O.RECON_PPM, q)
        for c in range(2, 14):
            lo = min(q[c - 1], q[c], q[c + 1])
            hi = max(q[c - 1], q[c], q[c + 1])
            assert lo - 1e-14 <= al[c] <= hi + 1e-14 and lo - 1e-14 <= ar[c] <= hi + 1e-14
            # the parabola has no interior extremum: q lies between the edge values ...
            assert (ar[c] - q[c]) * (q[c] - al[c]) >= -1e-14
            # ... and at a local extremum it is flat
            if (q[c + 1] - q[c]) * (q[c] - q[c - 1]) < 0:
                assert al[c] == q[c] and ar[c] == q[c]
        q2 = np.sort(q)
        al, ar = O.recon_line(O.RECON_PPM, q2)
        edges = np.ravel(np.column_stack([al[2:14], ar[2:14]]))
        assert np.all(np.diff(edges) >= -1e-13)


def test_source_vanishes_in_flat_space():
    d = _flat()
    p = np.array([1.0, 0.4, 0.3, -0.2, 0.1, 0.2, 0.1, 0.3])
    assert not np.any(O.source(d, p, 0, 0))


def _backward_error(d, prim, out, x1, x2):
    U0 = O.p2u_many(d, prim, x1, x2)
    U1 = O.p2u_many(d, out, x1, x2)
    scale = np.abs(U0[:, :5]).sum(axis=1)
    return np.abs(U1[:, :5] - U0[:, :5]).sum(axis=1) / scale


@pytest.mark.parametrize("a", [0.0, 0.9375])
def test_source_is_half_T_contracted_with_metric_derivatives(a):
    """Eq. for the source: with Gamma formed from the metric derivatives d_s g and the
    inverse metric, sqrt(-g) T^k_l Gamma^l_{nu k} = sqrt(-g) (1/2) T^{kl} d_nu g_{kl}
    (the form the FP64 cell update evaluates). Checked against the oracle's
    Christoffel contraction on random magnetised states, with d_s g by the same
    4th-order differences (h = 1e-3); the energy and phi-momentum sources vanish
    (stationary, axisymmetric metric)."""
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=a, gam=13.0 / 9.0)
    rng = np.random.default_rng(7)
    h = 1.0e-3
    for x1, x2 in [(math.log(1.6), 0.3), (math.log(7.0), 1.4), (math.log(30.0), 2.8)]:
        dg = np.zeros((4, 4, 4))
        for s_ in (1, 2):
            e = np.array([0.0, h if s_ == 1 else 0.0, h if s_ == 2 else 0.0])
            g = [O.geom(d, x1 + k * e[1], x2 + k * e[2])[0] for k in (2, 1, -1, -2)]
            dg[s_] = (-g[0] + 8.0 * g[1] - 8.0 * g[2] + g[3]) / (12.0 * h)
        gcov, gcon, gdet, _ = O.geom(d, x1, x2)
        for _ in range(20):
            pr = np.array([10 ** rng.uniform(-4, 0), 10 ** rng.uniform(-5, -1), *rng.normal(0, 0.5, 3),
                           *rng.normal(0, 0.05, 3)])
            ucon, ucov, bcon, bcov, bsq = O.state(d, pr, x1, x2)
            p = (13.0 / 9.0 - 1.0) * pr[1]
            eta = pr[0] + pr[1] + p + bsq
            T = eta * np.outer(ucon, ucon) + (p + 0.5 * bsq) * gcon - np.outer(bcon, bcon)
            q = O.source(d, pr, x1, x2)  # conserved slots: mass, energy, momentum 1..3, entropy
            scale = gdet * np.abs(T).max() * np.abs(dg).max()
            want = [0.5 * gdet * np.sum(T * dg[nu]) for nu in range(4)]
            for nu in range(4):
                assert abs(q[1 + nu] - want[nu]) <= 1e-12 * scale, (nu, q[1 + nu], want[nu])
            assert abs(q[1]) <= 1e-12 * scale and abs(q[4]) <= 1e-12 * scale
            assert q[0] == 0.0 and q[5] == 0.0


def test_con2prim_round_trip_random_states():
    """prim -> U -> prim with a 10% wrong guess over the whole range
    (rho 1e-6..1, u/rho 1e-4..1e2, Lorentz 1..50, sigma 0..100).
    The backward error |U(P_out) - U| / |U| is at round-off for moderate states;
    for sigma ~ 100 and Lorentz ~ 50 the recovery of utilde^i subtracts terms
    ~ sigma Gamma^2 larger than the result, which bounds it at ~1e-9."""
    d = _ks()
    prim, x1, x2 = W.random_states(20000, seed=5)
    U = O.p2u_many(d, prim, x1, x2)
    guess = prim.copy()
    guess[:, 0] *= 1.1
    guess[:, 1] *= 0.9
    guess[:, 2:5] *= 1.05
    out, st, it = O.c2p_many(d, U, prim[:, 5:8], x1, x2, guess)
    ok = st == 0
    assert ok.mean() > 0.999
    be = _backward_error(d, prim[ok], out[ok], x1[ok], x2[ok])
    assert be.max() < 1e-9

    prim2, x1b, x2b = W.random_states(4000, seed=7, lorentz_range=(1.0, 10.0), sigma_range=(0.0, 10.0),
                                      urho_range=(1e-2, 1e2))
    U2 = O.p2u_many(d, prim2, x1b, x2b)
    g2 = prim2.copy()
    g2[:, 0] *= 1.1
    g2[:, 1] *= 0.9
    out2, st2, it2 = O.c2p_many(d, U2, prim2[:, 5:8], x1b, x2b, g2)
    assert np.all(st2 == 0)
    be2 = _backward_error(d, prim2, out2, x1b, x2b)
    assert be2.max() < 2e-12
    rel = np.abs(out2[:, :5] - prim2[:, :5]) / np.abs(prim2[:, :5]).max(axis=1, keepdims=True)
    assert rel.max() < 1e-11
    assert it2.max() <= 12


def test_con2prim_entropy_backup_round_trip():
    """The entropy inversion alone recovers states whose U_kappa is consistent."""
    d = _ks()
    prim, x1, x2 = W.random_states(2000, seed=6, lorentz_range=(1.0, 10.0), sigma_range=(0.0, 10.0))
    U = O.p2u_many(d, prim, x1, x2)
    guess = prim.copy()
    guess[:, 0] *= 1.2
    out, st, it = O.c2p_many(d, U, prim[:, 5:8], x1, x2, guess, entropy_only=True)
    ok = st == 1
    assert ok.mean() > 0.995
    be = _backward_error(d, prim[ok], out[ok], x1[ok], x2[ok])
    assert np.quantile(be, 0.99) < 1e-12


def test_con2prim_recovers_energy_deficit_with_entropy():
    """Energy below what any u >= 0 allows: the energy inversion must not return it,
    the entropy backup must (Sec. 2.6)."""
    d = _ks()
    prim, x1, x2 = W.random_states(500, seed=8, urho_range=(1e-4, 1e-3), sigma_range=(0, 1),
                                   lorentz_range=(1.0, 2.0))
    U = O.p2u_many(d, prim, x1, x2)
    # remove 2x the internal energy density content from the energy slot
    U2 = U.copy()
    gdet = np.array([O.geom(d, a1, a2)[2] for a1, a2 in zip(x1, x2)])
    U2[:, 1] += 2.0 * prim[:, 1] * gdet * 5.0
    out, st, it = O.c2p_many(d, U2, prim[:, 5:8], x1, x2, prim)
    assert np.all(st != 0)
    ent = st == 1
    assert ent.mean() > 0.9
    assert np.all(out[ent, 1] > 0)
    assert np.allclose(out[ent, 0], prim[ent, 0], rtol=1e-3)
