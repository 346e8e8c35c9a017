"""Pins of the oracle's internal SMR (Sec. 3.3.2: phi-averaging next to the
pole so that polar cells stop limiting the time step): groups act as single
cells (identical primitives, uniform radial and theta faces, phi faces
linear inside a group), div B stays at round-off, the CFL step grows by the
group width where the pole limited it, and a uniform gas at rest stays at
rest to second order in flat spherical coordinates."""
import math

import numpy as np

import oracle as O
from paper_1912_10192_gb300 import workloads as W

NG = O.NG


def torus(smr, n=(32, 16, 16)):
    geo = W.torus_geometry(*n)
    prim, bf = W.torus_block(geo, seed=5)
    d = O.make_desc(*n, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3, metric=O.METRIC_KS, a=0.9375,
                    gam=13.0 / 9.0, cour=0.8, bc=(3, 3, 2, 2, 1, 1), smr=smr)
    return d, prim, bf


def _div(d, bf):
    f1 = bf[0][NG:NG + d.n3, NG:NG + d.n2, NG:NG + d.n1 + 1]
    f2 = bf[1][NG:NG + d.n3, NG:NG + d.n2 + 1, NG:NG + d.n1]
    f3 = bf[2][NG:NG + d.n3 + 1, NG:NG + d.n2, NG:NG + d.n1]
    return np.diff(f1, axis=2) / d.dx1 + np.diff(f2, axis=1) / d.dx2 + np.diff(f3, axis=0) / d.dx3


def test_groups_act_as_single_cells_and_div_b_stays_zero():
    d, prim, bf = torus(2)
    g = O.Grid(d)
    g.set(prim, bf)
    for _ in range(3):
        g.step()
    p, b = g.get()
    scale = np.abs(b).max() / min(d.dx1, d.dx2, d.dx3)
    assert np.abs(_div(d, b)).max() <= 1e-12 * scale
    for j, w in ((0, 4), (1, 2), (d.n2 - 1, 4), (d.n2 - 2, 2), (d.n2 // 2, 1)):
        row = p[:5, NG:NG + d.n3, NG + j, NG:NG + d.n1]  # (5, n3, n1)
        grp = row.reshape(5, d.n3 // w, w, d.n1)
        spread = np.abs(grp - grp[:, :, :1, :]).max()
        if w > 1:
            assert spread == 0.0, (j, w, spread)
            br = b[0][NG:NG + d.n3, NG + j, NG:NG + d.n1 + 1].reshape(d.n3 // w, w, d.n1 + 1)
            assert np.abs(br - br[:, :1, :]).max() == 0.0
            bp = b[2][NG:NG + d.n3 + 1, NG + j, NG:NG + d.n1]
            for k0 in range(0, d.n3, w):
                lin = bp[k0] + (bp[k0 + w] - bp[k0]) * (np.arange(w + 1)[:, None] / w)
                assert np.abs(bp[k0:k0 + w + 1] - lin).max() <= 1e-14 * np.abs(bp).max()
        else:  # an ungrouped row keeps its phi structure
            assert np.abs(row - row[:, :1, :]).max() > 0.0


def test_time_step_grows_where_the_pole_limits_it():
    dts = []
    for smr in (0, 2):
        d, prim, bf = torus(smr, n=(32, 32, 64))
        g = O.Grid(d)
        g.set(prim, bf)
        dts.append(g.dt())
    assert dts[1] > 1.5 * dts[0], dts


def test_axisymmetric_state_is_unchanged_by_the_grouping():
    """Without phi structure every group already is one cell: at a fixed dt the steps with and without
    internal SMR agree bitwise (a mixed-up row, face index or interpolation would break this)."""
    out = []
    for smr in (0, 2):
        geo = W.torus_geometry(32, 16, 16)
        prim, bf = W.torus_block(geo, seed=5, pert=0.0)
        d = O.make_desc(32, 16, 16, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3,
                        metric=O.METRIC_KS, a=0.9375, gam=13.0 / 9.0, cour=0.8, bc=(3, 3, 2, 2, 1, 1), smr=smr)
        g = O.Grid(d)
        g.set(prim, bf)
        for _ in range(3):
            g.step(0.05)
        out.append(g.get())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
