"""Pins of the oracle's Aitken-accelerated inversion (Sec. 2.6 names it beside
the 2-D Newton: Newman & Hamlin 2014): the pressure map against textbook
special-relativistic MHD states (the true pressure is its fixed point and
returns W = rho h Gamma^2 and v^2), the closed-form cubic root against a
polynomial root finder, round trips over the full range of states as for
Newton, and the convergence it gives from a cold start."""
import math

import numpy as np

import oracle as O
from paper_1912_10192_gb300 import workloads as W

GAM = 13.0 / 9.0


def _srmhd_state(rng):
    """A flat-space state: (rho, p, v, B) -> normal-frame E, S^2, (S.B)^2, B^2, D and W = rho h Gamma^2."""
    rho = 10.0 ** rng.uniform(-4, 0)
    p = rho * 10.0 ** rng.uniform(-3, 1)
    lor = 10.0 ** rng.uniform(0, math.log10(30.0))
    n = rng.normal(size=3)
    v = n / np.linalg.norm(n) * math.sqrt(1.0 - 1.0 / lor ** 2)
    B = rng.normal(size=3) * math.sqrt(rho) * 10.0 ** rng.uniform(-2, 1)
    h = 1.0 + GAM / (GAM - 1.0) * p / rho
    Wz = rho * h * lor ** 2
    vsq, vB, B2 = v @ v, v @ B, B @ B
    E = Wz - p + 0.5 * B2 + 0.5 * (vsq * B2 - vB ** 2)
    S = (Wz + B2) * v - vB * B
    return E, S @ S, (S @ B) ** 2, B2, rho * lor, Wz, vsq, p


def test_true_pressure_is_the_fixed_point_of_the_map():
    rng = np.random.default_rng(21)
    for _ in range(300):
        E, S2, T2, B2, D, Wz, vsq, p = _srmhd_state(rng)
        w, v, pn = O.nh_map(E, S2, T2, B2, D, GAM, p)
        assert abs(w - Wz) <= 1e-11 * (Wz + B2), (w, Wz)
        assert abs(v - vsq) <= 1e-10, (v, vsq)
        assert abs(pn - p) <= 1e-10 * (Wz + B2), (pn, p)


def test_cubic_root_is_the_largest_root():
    """For a trial p the map's W + B^2 is the largest real root of phi^3 - a phi^2 + d."""
    rng = np.random.default_rng(22)
    for _ in range(300):
        E, S2, T2, B2, D, Wz, vsq, p = _srmhd_state(rng)
        ptry = p * 10.0 ** rng.uniform(-1, 1)
        w, _, _ = O.nh_map(E, S2, T2, B2, D, GAM, ptry)
        a = E + ptry + 0.5 * B2
        d = 0.5 * (S2 * B2 - T2)
        roots = np.roots([1.0, -a, 0.0, d])
        big = max(r.real for r in roots if abs(r.imag) <= 1e-9 * a)
        assert abs((w + B2) - big) <= 1e-10 * a, (w + B2, big)


def test_aitken_round_trip_random_states():
    """prim -> U -> prim over the range of the Newton round-trip test, with the same guess."""
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=GAM, inversion=O.INV_AITKEN)
    prim, x1, x2 = W.random_states(20000, seed=5)
    U = O.p2u_many(d, prim, x1, x2)
    guess = prim.copy()
    guess[:, 0] *= 1.1
    guess[:, 1] *= 0.9
    guess[:, 2:5] *= 1.05
    out, st, it = O.c2p_many(d, U, prim[:, 5:8], x1, x2, guess)
    ok = st == 0
    assert ok.mean() > 0.999
    U1 = O.p2u_many(d, out[ok], x1[ok], x2[ok])
    be = np.abs(U1[:, :5] - U[ok, :5]).sum(axis=1) / np.abs(U[ok, :5]).sum(axis=1)
    assert be.max() < 1e-9
    # moderate states: round-off backward error, the primitives themselves, and few evaluations
    prim2, x1b, x2b = W.random_states(4000, seed=7, lorentz_range=(1.0, 10.0), sigma_range=(0.0, 10.0),
                                      urho_range=(1e-2, 1e2))
    U2 = O.p2u_many(d, prim2, x1b, x2b)
    g2 = prim2.copy()
    g2[:, 0] *= 1.1
    g2[:, 1] *= 0.9
    out2, st2, it2 = O.c2p_many(d, U2, prim2[:, 5:8], x1b, x2b, g2)
    assert np.all(st2 == 0)
    rel = np.abs(out2[:, :5] - prim2[:, :5]) / np.abs(prim2[:, :5]).max(axis=1, keepdims=True)
    assert rel.max() < 1e-11
    assert it2.max() <= 11 and it2.mean() < 8.0, (it2.max(), it2.mean())


def test_aitken_converges_from_a_cold_start():
    """From rho = D, u = 1e-3 D at rest (no usable guess) the pressure iteration reaches the root of
    every state of the wide range; Newton from the same start misses some."""
    dn = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=GAM)
    da = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=0.9375, gam=GAM, inversion=O.INV_AITKEN)
    prim, x1, x2 = W.random_states(5000, seed=9)
    U = O.p2u_many(dn, prim, x1, x2)
    cold = prim.copy()
    cold[:, 1] = 1e-3 * cold[:, 0]
    cold[:, 2:5] = 0.0
    _, stn, _ = O.c2p_many(dn, U, prim[:, 5:8], x1, x2, cold)
    outa, sta, ita = O.c2p_many(da, U, prim[:, 5:8], x1, x2, cold)
    assert np.all(sta == 0) and (stn == 0).mean() < 0.95
    rel = np.abs(outa[:, :2] - prim[:, :2]) / np.abs(prim[:, :2])
    assert np.quantile(rel[:, 0], 0.99) < 1e-9
