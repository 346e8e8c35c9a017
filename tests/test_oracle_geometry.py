"""Pins of the oracle's geometry (Sec. 2.2) against closed forms and sympy."""
import math

import numpy as np
import pytest

import oracle as O

POINTS = [(math.log(1.3), 0.4), (math.log(6.0), 1.2), (math.log(40.0), 2.9), (math.log(2.5), 0.05)]


def _desc(a):
    return O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_KS, a=a)


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9375])
def test_inverse_and_determinant(a):
    d = _desc(a)
    for x1, x2 in POINTS:
        gcov, gcon, gdet, alpha = O.geom(d, x1, x2)
        assert np.allclose(gcov @ gcon, np.eye(4), rtol=0, atol=1e-12 * np.abs(gcov).max())
        det = np.linalg.det(gcov)
        assert abs(det + gdet ** 2) <= 1e-11 * gdet ** 2
        assert abs(alpha - 1.0 / math.sqrt(-gcon[0, 0])) < 1e-15


def test_schwarzschild_textbook():
    """a = 0: ds^2 = -(1-2/r)dt^2 + (4/r)dt dr + (1+2/r)dr^2 + r^2 dOmega^2, with dr = r dx1."""
    d = _desc(0.0)
    for x1, x2 in POINTS:
        r = math.exp(x1)
        s2 = math.sin(x2) ** 2
        ref = np.zeros((4, 4))
        ref[0, 0] = -(1 - 2 / r)
        ref[0, 1] = ref[1, 0] = (2 / r) * r
        ref[1, 1] = (1 + 2 / r) * r * r
        ref[2, 2] = r * r
        ref[3, 3] = r * r * s2
        gcov, gcon, gdet, _ = O.geom(d, x1, x2)
        assert np.allclose(gcov, ref, rtol=1e-14, atol=1e-14)
        assert abs(gdet - r ** 3 * math.sin(x2)) < 1e-12 * r ** 3


def test_minkowski():
    d = O.make_desc(1, 1, 1, 0, 0, 0, 1, 1, 1, metric=O.METRIC_MINKOWSKI)
    gcov, gcon, gdet, alpha = O.geom(d, 0.3, 0.7)
    assert np.array_equal(gcov, np.diag([-1.0, 1, 1, 1])) and gdet == 1.0 and alpha == 1.0
    assert not np.any(O.conn(d, 0.3, 0.7))


@pytest.mark.parametrize("a", [0.0, 0.9375])
def test_connection_trace_identity(a):
    """Gamma^mu_{mu nu} = d_nu ln sqrt(-g), with sqrt(-g) = r Sigma sin(theta) in (log r, theta)."""
    d = _desc(a)
    for x1, x2 in POINTS:
        r = math.exp(x1)
        th = x2
        sig = r * r + a * a * math.cos(th) ** 2
        d1 = 1.0 + 2.0 * r * r / sig
        d2 = -2.0 * a * a * math.cos(th) * math.sin(th) / sig + math.cos(th) / math.sin(th)
        c = O.conn(d, x1, x2)
        tr = np.einsum("mmn->n", c)
        assert abs(tr[0]) < 1e-9 and abs(tr[3]) < 1e-9
        assert abs(tr[1] - d1) < 1e-9 * max(1, abs(d1))
        assert abs(tr[2] - d2) < 1e-8 * max(1, abs(d2))


def test_connection_vs_sympy():
    sp = pytest.importorskip("sympy")
    a = 0.9375
    t, x1, th, ph = sp.symbols("t x1 th ph")
    r = sp.exp(x1)
    sig = r ** 2 + a ** 2 * sp.cos(th) ** 2
    # Kerr in Kerr-Schild (t, r, th, ph) built from the line element, then dr = r dx1
    ks = sp.zeros(4, 4)
    ks[0, 0] = -(1 - 2 * r / sig)
    ks[0, 1] = ks[1, 0] = 2 * r / sig
    ks[0, 3] = ks[3, 0] = -2 * a * r * sp.sin(th) ** 2 / sig
    ks[1, 1] = 1 + 2 * r / sig
    ks[1, 3] = ks[3, 1] = -a * sp.sin(th) ** 2 * (1 + 2 * r / sig)
    ks[2, 2] = sig
    ks[3, 3] = sp.sin(th) ** 2 * (sig + a ** 2 * sp.sin(th) ** 2 * (1 + 2 * r / sig))
    J = sp.diag(1, r, 1, 1)
    g = J.T * ks * J
    X = [t, x1, th, ph]
    dg = [[[sp.diff(g[m, n], X[s]) for n in range(4)] for m in range(4)] for s in range(4)]
    d = _desc(a)
    for (xv1, xv2) in POINTS[:3]:
        sub = {x1: xv1, th: xv2}
        gnum = np.array(g.subs(sub).evalf(), dtype=float)
        ginv = np.linalg.inv(gnum)
        dgn = np.array([[[float(dg[s][m][n].subs(sub).evalf()) for n in range(4)] for m in range(4)]
                        for s in range(4)])
        ref = 0.5 * (np.einsum("lk,mkn->lmn", ginv, dgn) + np.einsum("lk,nkm->lmn", ginv, dgn)
                     - np.einsum("lk,kmn->lmn", ginv, dgn))
        c = O.conn(d, xv1, xv2)
        scale = np.abs(ref).max()
        assert np.abs(c - ref).max() < 1e-9 * scale
