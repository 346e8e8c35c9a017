"""Pins of the oracle's flat spherical metric (flat space in the log-r
spherical coordinates of the Kerr-Schild grid, used by the off-centre
explosion through the pole of Sec. 6): the metric and its determinant in
closed form, the connection against the Christoffel symbols of flat space in
(log r, theta, phi) worked out by hand, and a uniform gas at rest kept at
rest up to a truncation error that converges at second order (the pressure
flux divergence against the geometric source)."""
import math

import numpy as np

import oracle as O

NG = O.NG


def _desc(n1=1, n2=1, n3=1, x1min=0.0, x2min=0.0, dx1=1.0, dx2=1.0, dx3=1.0, bc=(0, 0, 0, 0, 1, 1)):
    return O.make_desc(n1, n2, n3, x1min, x2min, 0.0, dx1, dx2, dx3, metric=O.METRIC_SPHERICAL, a=0.9,
                       gam=5.0 / 3.0, cour=0.5, bc=bc, floors=0)


def test_metric_and_connection_closed_forms():
    d = _desc()
    for x1, th in ((0.3, 0.7), (2.0, 1.9), (-0.5, 0.2)):
        r, s, c = math.exp(x1), math.sin(th), math.cos(th)
        gcov, gcon, gdet, alpha = O.geom(d, x1, th)
        assert np.allclose(gcov, np.diag([-1.0, r * r, r * r, r * r * s * s]), rtol=1e-15, atol=0)
        assert np.allclose(gcon @ gcov, np.eye(4), rtol=0, atol=1e-14)
        assert abs(gdet - r ** 3 * s) <= 1e-14 * r ** 3 and alpha == 1.0
        G = O.conn(d, x1, th)  # G[l, m, n] = Gamma^l_{mn}
        want = np.zeros((4, 4, 4))
        want[1, 1, 1] = 1.0
        want[1, 2, 2] = -1.0
        want[1, 3, 3] = -s * s
        want[2, 1, 2] = want[2, 2, 1] = 1.0
        want[2, 3, 3] = -s * c
        want[3, 1, 3] = want[3, 3, 1] = 1.0
        want[3, 2, 3] = want[3, 3, 2] = c / s
        assert np.abs(G - want).max() < 1e-9, np.abs(G - want).max()


def _static_error(n):
    """One step of a uniform gas at rest on r in [2, 4], theta in [0.8, 2.3]: max |utilde| after the step."""
    x1a, x1b, tha, thb = math.log(2.0), math.log(4.0), 0.8, 2.3
    d = _desc(n, n, 4, x1a, tha, (x1b - x1a) / n, (thb - tha) / n, 0.1)
    prim = np.zeros((8, 4 + 2 * NG, n + 2 * NG, n + 2 * NG))
    prim[0] = 1.0
    prim[1] = 1.0
    g = O.Grid(d)
    g.set(prim, np.zeros((3,) + prim.shape[1:]))
    dt = 0.1 * (x1b - x1a) / n * 2.0
    g.step(dt)
    p, _ = g.get()
    s = (slice(NG + 1, NG + 3), slice(NG + 2, NG + n - 2), slice(NG + 2, NG + n - 2))
    return max(np.abs(p[v][s]).max() for v in (2, 3)) / dt


def test_uniform_gas_at_rest_stays_at_rest_to_second_order():
    e = [_static_error(n) for n in (8, 16)]
    assert e[0] < 1e-2 and 3.2 < e[0] / e[1] < 4.8, e
