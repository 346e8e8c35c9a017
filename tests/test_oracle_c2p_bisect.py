"""Brute-force pin of the oracle's energy inversion (Sec. 2.6; the unknowns
(W, v^2) and the two equations of Noble et al. 2006).

From each conserved state the test forms the normal-frame scalars itself
(D, Q.n, Qt^2, Q.B, B^2 from the definitions, in long double), eliminates
v^2 with the momentum equation (v^2 is a closed form of W), and finds every
root of the remaining energy equation in W on the admissible branch
(0 <= v^2 < 1) by scanning for sign changes on a logarithmic grid and
bisecting in long double. That is a different algorithm from the oracle's
two-dimensional Newton iteration, and it checks:

* uniqueness: exactly one admissible root per state over the sampled law;
* the root is the W = (rho + u + p) Gamma^2 of the primitives the conserved
  state was formed from (this pins the test's own scalars). The conserved
  state is that W's only up to the rounding of the FP64 prim -> cons map,
  which relativistic, cold states amplify (about Gamma^2 over the thermal
  fraction of W): measured up to 9e-11 relative over the full law, so the
  bar is 1e-9 there and round-off for moderate states;
* the oracle's converged W equals the root.

Tolerance of the last check: a root of f(W) = 0 evaluated in floating point
is uncertain by about eps * sum|terms of f| / |W f'(W)| (the rounding of f
near the root over its slope); the bar is 64 times that condition number
times the double unit round-off, state by state (measured: at most 1.7).
"""
import math

import numpy as np

import oracle as O
from paper_1912_10192_gb300 import workloads as W

LD = np.longdouble
EPS = np.finfo(np.float64).eps


def scalars(d, U, B, x1, x2):
    n = U.shape[0]
    out = {k: np.zeros(n, LD) for k in ("D", "Qn", "Qt2", "QB", "B2")}
    for s in range(n):
        gcov, gcon, gdet, alpha = O.geom(d, x1[s], x2[s])
        gcov, gcon = gcov.astype(LD), gcon.astype(LD)
        sg, al = LD(gdet), LD(alpha)
        u = U[s].astype(LD)
        D = al * u[0] / sg                                     # rho Gamma = alpha rho u^t
        Qcov = np.array([al * (u[1] - u[0]) / sg, al * u[2] / sg, al * u[3] / sg, al * u[4] / sg], LD)
        Qcon = gcon @ Qcov
        Qn = -al * Qcon[0]                                     # Q_mu n^mu, n_mu = (-alpha, 0, 0, 0)
        Bn = np.concatenate([[LD(0)], al * B[s].astype(LD)])
        out["D"][s] = D
        out["Qn"][s] = Qn
        out["Qt2"][s] = Qcov @ Qcon + Qn * Qn
        out["QB"][s] = Qcov @ Bn
        out["B2"][s] = Bn @ gcov @ Bn
    return out


def vsq_of_w(S, w):
    return (S["Qt2"] + S["QB"] ** 2 * (S["B2"] + 2 * w) / (w * w)) / (S["B2"] + w) ** 2


def terms(S, w, gam):
    """The terms of the energy equation f(W) = sum(terms) = 0 with v^2 eliminated."""
    v2 = vsq_of_w(S, w)
    sq = np.sqrt(np.maximum(LD(1) - v2, LD(0)))
    gf = LD(gam - 1.0) / LD(gam)
    return [-S["B2"] * (1 + v2) / 2, S["QB"] ** 2 / (2 * w * w), -w, gf * w * (1 - v2), -gf * S["D"] * sq, -S["Qn"]]


def f_of_w(S, w, gam):
    return sum(terms(S, w, gam))


def w_branch_start(S):
    """Smallest W with v^2(W) < 1 (v^2 falls monotonically with W)."""
    lo = np.full_like(S["D"], LD(1e-30))
    hi = np.maximum(S["D"], LD(1e-30))
    while np.any(vsq_of_w(S, hi) >= 1):
        hi = np.where(vsq_of_w(S, hi) >= 1, hi * 4, hi)
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        big = vsq_of_w(S, mid) >= 1
        lo = np.where(big, mid, lo)
        hi = np.where(big, hi, mid)
    return hi


def all_roots(S, gam, npts=600):
    w0 = w_branch_start(S) * (1 + LD(1e-15))
    w1 = np.maximum(LD(1e4) * w0, LD(10) * (-S["Qn"]))
    grid = [w0 * (w1 / w0) ** (LD(m) / (npts - 1)) for m in range(npts)]
    fv = [f_of_w(S, w, gam) for w in grid]
    roots = [[] for _ in range(len(w0))]
    for m in range(npts - 1):
        ch = np.nonzero(np.sign(fv[m]) * np.sign(fv[m + 1]) < 0)[0]
        for s in ch:
            a, b, fa = grid[m][s], grid[m + 1][s], fv[m][s]
            Ss = {k: v[s:s + 1] for k, v in S.items()}
            for _ in range(200):
                c = (a + b) / 2
                fc = f_of_w(Ss, np.array([c]), gam)[0]
                if (fc > 0) == (fa > 0):
                    a, fa = c, fc
                else:
                    b = c
            roots[s].append((a + b) / 2)
    return roots


def w_of_prim(d, prim, x1, x2, gam):
    n = prim.shape[0]
    w = np.zeros(n, LD)
    for s in range(n):
        gcov, _, _, _ = O.geom(d, x1[s], x2[s])
        ut = prim[s, 2:5].astype(LD)
        g2 = 1 + ut @ gcov[1:, 1:].astype(LD) @ ut
        rho, u = LD(prim[s, 0]), LD(prim[s, 1])
        w[s] = (rho + u + LD(gam - 1.0) * u) * g2
    return w


def condition(S, w, gam):
    """sum|terms| / |W f'(W)| at the root (f' by a central difference in long double)."""
    h = w * LD(1e-7)
    fp = (f_of_w(S, w + h, gam) - f_of_w(S, w - h, gam)) / (2 * h)
    mag = sum(np.abs(t) for t in terms(S, w, gam))
    return mag / np.abs(w * fp)


def run(metric, a, gam, n, seed, **law):
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=metric, a=a, gam=gam)
    prim, x1, x2 = W.random_states(n, seed=seed, a=a if metric == O.METRIC_KS else 0.0, **law)
    if metric == O.METRIC_MINKOWSKI:
        x1 = np.zeros(n)
        x2 = np.full(n, 0.5 * math.pi)
        # flat space: the drawn utilde^i and B^i are taken as Cartesian components (any utilde is a
        # valid velocity; the Lorentz factors and magnetisations shift with the metric)
    U = O.p2u_many(d, prim, x1, x2)
    guess = prim.copy()
    guess[:, 0] *= 1.05
    guess[:, 1] *= 0.95
    guess[:, 2:5] *= 1.02
    po, st, _ = O.c2p_many(d, U, prim[:, 5:8], x1, x2, guess)
    S = scalars(d, U, prim[:, 5:8], x1, x2)
    roots = all_roots(S, gam)
    return d, prim, x1, x2, po, st, S, roots


def check(metric, a, gam, n, seed, true_bar, **law):
    d, prim, x1, x2, po, st, S, roots = run(metric, a, gam, n, seed, **law)
    nroots = np.array([len(r) for r in roots])
    assert np.all(nroots == 1), np.bincount(nroots)
    wb = np.array([r[0] for r in roots], LD)
    wt = w_of_prim(d, prim, x1, x2, gam)
    kappa = condition(S, wb, gam)
    bar = 64 * EPS * kappa + 4 * EPS
    rel_true = np.abs(wb - wt) / wb
    assert np.all(rel_true <= true_bar), float(rel_true.max())
    ok = st == 0
    assert ok.mean() > 0.97, ok.mean()
    wo = w_of_prim(d, po[ok], x1[ok], x2[ok], gam)
    rel_ora = np.abs(wo - wb[ok]) / wb[ok]
    assert np.all(rel_ora <= bar[ok]), float((rel_ora / bar[ok]).max())
    return rel_ora, bar[ok], kappa


def test_inversion_root_is_the_unique_bisected_root_kerr_schild():
    rel, bar, kappa = check(O.METRIC_KS, 0.9375, 13.0 / 9.0, 1500, seed=71, true_bar=1e-9)
    # the law reaches ill-conditioned states (sigma ~ 100, Lorentz ~ 50): the bar is not vacuous there
    assert kappa.max() > 1e3 and np.median(kappa) < 1e2


def test_inversion_root_is_the_unique_bisected_root_flat_space():
    check(O.METRIC_MINKOWSKI, 0.0, 5.0 / 3.0, 1000, seed=72, true_bar=1e-9)


def test_inversion_root_moderate_states():
    rel, bar, kappa = check(O.METRIC_KS, 0.5, 4.0 / 3.0, 1000, seed=73, true_bar=1e-13,
                            lorentz_range=(1.0, 5.0), sigma_range=(0.0, 5.0))
    # well-conditioned states: the oracle's W is the root to a few units of round-off
    assert np.all(rel <= 64 * EPS * kappa + 4 * EPS) and float(np.median(rel)) < 1e-15
