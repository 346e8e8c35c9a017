"""Pins of the oracle's internal SMR (Sec. 3.3.2: phi-averaging next to the
pole so that polar cells stop limiting the time step): groups act as single
cells (identical primitives; the field changes as a wide cell's: uniform
changes of the radial and theta faces, linear changes of the phi faces inside
a group), div B stays at round-off, a state mirror-symmetric in phi stays so
(the group means and interpolations treat both ends of a group alike), the
CFL step grows by the group width where the pole limited it, and an
axisymmetric state is stepped bitwise as without grouping."""
import math

import numpy as np

import oracle as O
from paper_1912_10192_gb300 import workloads as W

from helpers import polar_field_desc

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
    """The torus with a field through the poles that varies in phi: after each step the grouped cells
    hold identical primitives, each group's x1- and x2-faces changed by one amount and its inner
    x3-faces by amounts linear between its outer ones, div B at round-off."""
    d, prim, bf = torus(2)
    polar_field_desc(bf, d)
    g = O.Grid(d)
    g.set(prim, bf)
    scale = np.abs(bf).max() / min(d.dx1, d.dx2, d.dx3)
    _, b0 = g.get()
    for _ in range(3):
        g.step()
        p, b = g.get()
        assert np.abs(_div(d, b)).max() <= 1e-12 * scale
        db = b - b0
        for j, w in ((0, 4), (1, 2), (d.n2 - 1, 4), (d.n2 - 2, 2), (d.n2 // 2, 1)):
            row = p[:5, NG:NG + d.n3, NG + j, NG:NG + d.n1]  # (5, n3, n1)
            grp = row.reshape(5, d.n3 // w, w, d.n1)
            if w == 1:  # an ungrouped row keeps its phi structure
                assert np.abs(row - row[:, :1, :]).max() > 0.0
                continue
            assert np.abs(grp - grp[:, :, :1, :]).max() == 0.0, (j, w)
            jf = j + 1 if j < d.n2 // 2 else j  # the x2-face away from the pole
            for m, jj, e in ((0, j, d.n1 + 1), (1, jf, d.n1)):
                ch = db[m][NG:NG + d.n3, NG + jj, NG:NG + e].reshape(d.n3 // w, w, e)
                assert np.abs(ch - ch[:, :1, :]).max() <= 1e-13 * np.abs(db[m]).max(), (j, w, m)
            c3 = db[2][NG:NG + d.n3 + 1, NG + j, NG:NG + d.n1]
            for k0 in range(0, d.n3, w):
                lin = c3[k0] + (c3[k0 + w] - c3[k0]) * (np.arange(w + 1)[:, None] / w)
                assert np.abs(c3[k0:k0 + w + 1] - lin).max() <= 1e-13 * np.abs(db[2]).max(), (j, w, k0)
        b0 = b


def test_phi_mirror_symmetric_state_stays_symmetric():
    """Flat space, an explosion centred on the plane phi = 0 next to the axis and the field through the
    poles (even in phi): the scheme is mirror-symmetric in phi (rho, u, utilde^1,2 and the x1-, x2-face
    fluxes even; utilde^3 and the x3-face fluxes odd) and so are the group means and linear
    interpolations of internal SMR; a rule that treats the two ends of a group differently breaks it."""
    n1, n2, n3 = 24, 16, 16
    x1a, x1b = math.log(2.0), math.log(40.0)
    d = O.make_desc(n1, n2, n3, x1a, 0.0, 0.0, (x1b - x1a) / n1, math.pi / n2, 2.0 * math.pi / n3,
                    metric=O.METRIC_SPHERICAL, gam=5.0 / 3.0, cour=0.8, bc=(3, 3, 2, 2, 1, 1), floors=0, smr=2)
    blk = dict(n1=n1, n2=n2, n3=n3, x1min=d.x1min, x2min=d.x2min, x3min=d.x3min, dx1=d.dx1, dx2=d.dx2, dx3=d.dx3)
    (prim, bf), = W.explosion_blocks([blk], centre=(1.5, 0.0, 8.0), gam=5.0 / 3.0)
    polar_field_desc(bf, d, B0=1e-4)
    g = O.Grid(d)
    g.set(prim, bf)
    for _ in range(4):
        g.step()
    p, b = g.get()
    c = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
    for q, sgn in ((0, 1), (1, 1), (2, 1), (3, 1), (4, -1)):
        x = p[q][c]
        assert np.abs(x - sgn * x[::-1]).max() <= 1e-10 * np.abs(x).max(), q
    for m, sgn in ((0, 1), (1, 1)):
        e = [n3, n2, n1]
        e[2 - m] += 1
        x = b[m][NG:NG + e[0], NG:NG + e[1], NG:NG + e[2]]
        assert np.abs(x - sgn * x[::-1]).max() <= 1e-10 * np.abs(x).max(), m
    x = b[2][NG:NG + n3 + 1, NG:NG + n2, NG:NG + n1]  # face k mirrors to face n3 - k
    assert np.abs(x + x[::-1]).max() <= 1e-10 * np.abs(x).max()
    assert np.abs(x[:, :4]).max() > 1e-3 * np.abs(x).max()  # the grouped rows carry phi field


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
