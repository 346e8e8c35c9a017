"""Pins of the oracle's PPM shock flattener (Sec. 2.1: PPM with an optional
flattener that lowers the order of the reconstruction at shocks, Colella &
Woodward 1984): the coefficient on profiles whose value follows from its
definition by hand, the reconstruction at the coefficient's two ends, and a
relativistic shock problem against its exact solution."""
import numpy as np
import pytest

import oracle as O
from paper_1912_10192_gb300 import workloads as W

NG = O.NG
GAM = 5.0 / 3.0


def _coef(p, w):
    return O.flatten_line(GAM, np.asarray(p, float) / (GAM - 1.0), np.asarray(w, float))


def test_sharp_shock_flattens_the_two_cells_beside_it():
    # one jump between cells 4 and 5 of a converging flow: for both, p(c+1) - p(c-1) = p(c+2) - p(c-2)
    p = [1.0] * 5 + [10.0] * 5
    w = [0.5] * 5 + [-0.5] * 5
    f = _coef(p, w)
    assert f.tolist() == [0, 0, 0, 0, 1, 1, 0, 0, 0, 0]


def test_smooth_and_expanding_and_weak_profiles_are_not_flattened():
    conv = np.linspace(0.5, -0.5, 12)
    # a linear pressure ramp: p(c+2) - p(c-2) = 2 (p(c+1) - p(c-1)), ratio 1/2 below 3/4
    assert not _coef(1.0 + np.arange(12.0), conv).any()
    # the sharp jump of the first test in an expanding flow
    assert not _coef([1.0] * 5 + [10.0] * 5, -np.linspace(0.5, -0.5, 10)).any()
    # a jump of 30% of the lower pressure (below the 0.33 threshold), and one of 34% (above)
    assert not _coef([1.0] * 5 + [1.30] * 5, np.linspace(0.5, -0.5, 10)).any()
    assert _coef([1.0] * 5 + [1.34] * 5, np.linspace(0.5, -0.5, 10))[4:6].tolist() == [1.0, 1.0]


def test_partial_coefficient_and_two_cell_shock():
    conv = np.linspace(0.5, -0.5, 7)
    # at c = 3: dp1 = p4 - p2 = 4, dp2 = p5 - p1 = 5: f = 10 (0.8 - 0.75) = 0.5
    f = _coef([1.0, 1.0, 2.0, 4.0, 6.0, 6.0, 6.0], conv)
    assert abs(f[3] - 0.5) < 1e-14
    # a shock spread over two cells: its middle cell has ratio 1, its edges ratio 1/2
    f = _coef([1.0, 1.0, 1.0, 4.0, 7.0, 7.0, 7.0], conv)
    assert f.tolist() == [0, 0, 0, 1, 0, 0, 0]


def test_narrow_pressure_peak_is_flattened_whatever_the_rounding_noise():
    """Two streams meeting: a two-cell pressure peak. For the peak cells p(c+2) - p(c-2) is zero,
    or rounding noise after a step; the coefficient (magnitude ratio) is 1 on the peak and its
    flanks either way, and 0 away from it."""
    conv = np.linspace(0.5, -0.5, 10)
    base = np.array([0.01] * 4 + [0.7, 0.7] + [0.01] * 4)
    want = [0, 0, 0, 1, 1, 1, 1, 0, 0, 0]
    assert _coef(base, conv).tolist() == want
    rng = np.random.default_rng(11)
    for _ in range(20):
        noisy = base * (1.0 + 1e-15 * rng.standard_normal(10))
        assert _coef(noisy, conv).tolist() == want


def test_reconstruction_at_the_coefficient_ends():
    rng = np.random.default_rng(5)
    q = np.cumsum(rng.normal(size=40))
    al, ar = O.recon_line(O.RECON_PPM, q)
    fl, fr = O.recon_line_flat(q, np.zeros_like(q))
    assert np.array_equal(al[2:-2], fl[2:-2]) and np.array_equal(ar[2:-2], fr[2:-2])
    fl, fr = O.recon_line_flat(q, np.ones_like(q))  # f = 1: piecewise constant (first order)
    assert np.array_equal(fl[2:-2], q[2:-2]) and np.array_equal(fr[2:-2], q[2:-2])
    # a linear profile has exact interface values c +- 1/2; f blends them toward the cell value
    lin = np.arange(20.0)
    f = np.linspace(0.0, 1.0, 20)
    fl, fr = O.recon_line_flat(lin, f)
    c = np.arange(2, 18)
    assert np.allclose(fl[c], lin[c] - 0.5 * (1.0 - f[c]), rtol=0, atol=1e-13)
    assert np.allclose(fr[c], lin[c] + 0.5 * (1.0 - f[c]), rtol=0, atol=1e-13)


def _riemann(n1, left, right, flatten, T=0.4):
    import srhd_exact as X
    prim, bf = W.riemann_block(n1, left, right, gam=GAM)
    d = O.make_desc(n1, 4, 4, 0.0, 0.0, 0.0, 1.0 / n1, 1.0, 1.0, metric=O.METRIC_MINKOWSKI, gam=GAM, cour=0.5,
                    recon=O.RECON_PPM, riemann=O.FLUX_HLL, bc=(0, 0, 1, 1, 1, 1), floors=0, flatten=flatten)
    g = O.Grid(d)
    g.set(prim, bf)
    t = 0.0
    while t < T - 1e-13:
        t += g.step(min(g.dt(), T - t))
    p, _ = g.get()
    L, R = X.State(*left, GAM), X.State(*right, GAM)
    pstar = X.solve(L, R)[0]
    xc = (np.arange(n1) + 0.5) / n1
    ex = np.array([X.sample(L, R, (x - 0.5) / T) for x in xc])
    row = (slice(None), NG + 1, NG + 1, slice(NG, NG + n1))
    rho, pr, ut = p[0][row[1:]], (GAM - 1.0) * p[1][row[1:]], p[2][row[1:]]
    v = ut / np.sqrt(1.0 + ut * ut)
    err = [np.abs(a - ex[:, m]).mean() for m, a in enumerate((rho, pr, v))]
    return pr.max() / pstar, err


@pytest.mark.parametrize("vc", [0.9, 0.6])
def test_flattener_removes_post_shock_oscillations_of_colliding_streams(vc):
    """Two cold streams at +-vc collide at x = 0.5: two shocks run outward and leave a uniform hot
    state at the exact p*. Plain PPM rings behind the shocks (pressure overshoots p* by several per
    cent); with the flattener the overshoot is below 2% and the L1 pressure error drops."""
    p0 = 0.01 if vc > 0.8 else 0.1
    left, right = (1.0, p0, vc), (1.0, p0, -vc)
    over0, e0 = _riemann(200, left, right, 0)
    over1, e1 = _riemann(200, left, right, 1)
    assert over0 > 1.05 and over1 < 1.02, (over0, over1)
    assert e1[1] < 0.85 * e0[1], (e0, e1)
    assert e1[2] < e0[2], (e0, e1)
