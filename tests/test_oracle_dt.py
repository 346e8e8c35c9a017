"""Pins of the oracle's CFL time step (Sec. 2.1: dt = C0 / max over cells of
sum_i v_f^i / dx^i, the footnote of Sec. 3.3 for the fastest speed per
direction) against closed forms that do not go through the oracle's
dispersion relation:

* gas at rest in flat Cartesian space: every direction's fastest speed is the
  fluid-frame magnetosonic speed c, so dt = C0 / (c (1/dx1 + 1/dx2 + 1/dx3));
  unequal cell widths separate "sum over directions" from "max over them";
* a boosted gas: along the flow the relativistic velocity addition
  (|v| + c)/(1 + |v| c), across it c sqrt(1 - v^2) / sqrt(1 - v^2 c^2) (the
  transverse characteristic of special-relativistic hydrodynamics); a flow
  toward -x makes |v-| the larger speed, so a "|v+| only" slip fails;
* a hot cell in a cold box sets dt alone (max over cells);
* gas at rest in flat space in the log-r spherical coordinates: the speeds
  in (x1 = log r, theta, phi) are c/r, c/r and c/(r sin theta), largest in
  the innermost polar cell.
"""
import math

import numpy as np
import pytest

import oracle as O

NG = O.NG
C0 = 0.8


def sound_speed2(rho, u, gam):
    p = (gam - 1.0) * u
    return gam * p / (rho + u + p)


def fast_speed2(rho, u, gam, b2):
    """Fluid-frame fast speed of the paper's approximation: vA^2 + cs^2 (1 - vA^2)."""
    p = (gam - 1.0) * u
    w = rho + u + p
    va2 = b2 / (b2 + w)
    cs2 = gam * p / w
    return va2 + cs2 * (1.0 - va2)


def box(n, dx, metric=O.METRIC_MINKOWSKI, gam=5.0 / 3.0, x0=(0.0, 0.0, 0.0), bc=(O.BC_PERIODIC,) * 6):
    d = O.make_desc(n[0], n[1], n[2], x0[0], x0[1], x0[2], dx[0], dx[1], dx[2], metric=metric, gam=gam,
                    cour=C0, bc=bc, floors=0)
    shp = (n[2] + 2 * NG, n[1] + 2 * NG, n[0] + 2 * NG)
    return d, np.zeros((8,) + shp), np.zeros((3,) + shp)


def grid_dt(d, prim, bf):
    g = O.Grid(d)
    g.set(prim, bf)
    return g.dt()


DX = (0.1, 0.025, 0.04)   # unequal widths: sum and max over directions differ


def test_gas_at_rest_flat():
    gam = 5.0 / 3.0
    d, prim, bf = box((6, 5, 4), DX, gam=gam)
    prim[0], prim[1] = 1.3, 0.7
    c = math.sqrt(sound_speed2(1.3, 0.7, gam))
    expect = C0 / (c * sum(1.0 / h for h in DX))
    assert abs(grid_dt(d, prim, bf) - expect) <= 1e-14 * expect


def test_magnetised_gas_at_rest_flat():
    """A uniform face field along x: b^mu = (0, B) at rest, b^2 = B^2; the
    approximate fast speed is isotropic."""
    gam = 4.0 / 3.0
    d, prim, bf = box((6, 5, 4), DX, gam=gam)
    prim[0], prim[1] = 0.5, 0.2
    B = 0.9
    bf[0] = B
    c = math.sqrt(fast_speed2(0.5, 0.2, gam, B * B))
    expect = C0 / (c * sum(1.0 / h for h in DX))
    assert abs(grid_dt(d, prim, bf) - expect) <= 1e-14 * expect
    # the magnetosonic speed is faster than sound: a slip that drops b^2 gives a larger dt
    assert expect < C0 / (math.sqrt(sound_speed2(0.5, 0.2, gam)) * sum(1.0 / h for h in DX))


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("v", [-0.6, 0.95])
def test_boosted_gas_flat(axis, v):
    gam = 5.0 / 3.0
    d, prim, bf = box((6, 5, 4), DX, gam=gam)
    rho, u = 1.0, 2.0
    prim[0], prim[1] = rho, u
    lorentz = 1.0 / math.sqrt(1.0 - v * v)
    prim[2 + axis] = lorentz * v            # utilde^i = Gamma v^i in flat space
    c = math.sqrt(sound_speed2(rho, u, gam))
    along = (abs(v) + c) / (1.0 + abs(v) * c)
    across = c * math.sqrt(1.0 - v * v) / math.sqrt(1.0 - v * v * c * c)
    rate = sum((along if m == axis else across) / DX[m] for m in range(3))
    expect = C0 / rate
    assert abs(grid_dt(d, prim, bf) - expect) <= 1e-13 * expect


def test_hot_cell_sets_the_step():
    gam = 5.0 / 3.0
    d, prim, bf = box((8, 6, 4), DX, gam=gam)
    prim[0], prim[1] = 1.0, 1e-3
    hot = (NG + 2, NG + 3, NG + 5)
    prim[1][hot] = 50.0
    c = math.sqrt(sound_speed2(1.0, 50.0, gam))
    expect = C0 / (c * sum(1.0 / h for h in DX))
    assert abs(grid_dt(d, prim, bf) - expect) <= 1e-14 * expect


def test_gas_at_rest_flat_spherical():
    """Flat space in (log r, theta, phi): g^11 = 1/r^2, g^22 = 1/r^2,
    g^33 = 1/(r sin theta)^2, so v_f^i = c sqrt(g^ii); the largest rate is in
    the innermost cell next to a pole."""
    gam = 13.0 / 9.0
    n = (8, 8, 6)
    x1min, x1max = math.log(2.0), math.log(6.0)
    dx = ((x1max - x1min) / n[0], math.pi / n[1], 2 * math.pi / n[2])
    bc = (O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_POLAR, O.BC_POLAR, O.BC_PERIODIC, O.BC_PERIODIC)
    d, prim, bf = box(n, dx, metric=O.METRIC_SPHERICAL, gam=gam, x0=(x1min, 0.0, 0.0), bc=bc)
    prim[0], prim[1] = 1.0, 0.4
    c = math.sqrt(sound_speed2(1.0, 0.4, gam))
    best = 0.0
    for j in range(n[1]):
        th = (j + 0.5) * dx[1]
        for i in range(n[0]):
            r = math.exp(x1min + (i + 0.5) * dx[0])
            best = max(best, c / r * (1.0 / dx[0] + 1.0 / dx[1] + 1.0 / (math.sin(th) * dx[2])))
    expect = C0 / best
    assert abs(grid_dt(d, prim, bf) - expect) <= 1e-13 * expect
