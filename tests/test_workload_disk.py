"""The tilted thin-disk initial state: divergence-free face field, polar-axis
faces without flux, the stated plasma beta, density normalisation, the tilt
of the density maximum and the Keplerian rotation about the tilted axis."""
import math

import numpy as np

import oracle as O
from paper_1912_10192_gb300 import workloads as W

NG = 3


def _case(n1=56, n2=24, n3=48):
    geo = W.disk_geometry(n1, n2, n3)
    prim, bf = W.tilted_disk_block(geo)
    return geo, prim, bf


def test_face_field_is_divergence_free_and_axis_faces_empty():
    geo, prim, bf = _case()
    n1, n2, n3 = geo.n1, geo.n2, geo.n3
    b1 = bf[0][NG:NG + n3, NG:NG + n2, NG:NG + n1 + 1]
    b2 = bf[1][NG:NG + n3, NG:NG + n2 + 1, NG:NG + n1]
    b3 = bf[2][NG:NG + n3, NG:NG + n2, NG:NG + n1]
    b3p = np.concatenate([b3, b3[:1]], axis=0)  # periodic phi
    div = ((b1[:, :, 1:] - b1[:, :, :-1]) / geo.dx1 + (b2[:, 1:, :] - b2[:, :-1, :]) / geo.dx2
           + (b3p[1:] - b3p[:-1]) / geo.dx3)
    scale = max(np.abs(b1).max(), np.abs(b2).max(), np.abs(b3).max()) / min(geo.dx1, geo.dx2, geo.dx3)
    assert np.abs(div).max() <= 1e-13 * scale
    assert np.all(b2[:, 0, :] == 0.0) and np.all(b2[:, -1, :] == 0.0)
    assert np.abs(b3).max() > 0.1 * np.abs(b1).max()  # the tilt gives the field components in every direction


def test_density_peak_lies_in_the_tilted_midplane():
    geo, prim, _ = _case()
    n1, n2, n3 = geo.n1, geo.n2, geo.n3
    rho = prim[0][NG:NG + n3, NG:NG + n2, NG:NG + n1]
    assert 0.9 < rho.max() <= 1.0 + 1e-12
    th = geo.x2min + (np.arange(n2) + 0.5) * geo.dx2
    ph = geo.x3min + (np.arange(n3) + 0.5) * geo.dx3
    tl = math.radians(65.0)
    nvec = np.array([0.0, -math.sin(tl), math.cos(tl)])
    k, j, i = np.unravel_index(np.argmax(rho), rho.shape)
    rhat = np.array([math.sin(th[j]) * math.cos(ph[k]), math.sin(th[j]) * math.sin(ph[k]), math.cos(th[j])])
    # the maximum sits within a cell or so of the tilted midplane, not the grid equator
    assert abs(rhat @ nvec) < 2.0 * geo.dx2
    # the disk reaches theta far from pi/2 (tilt 65 deg): the density maximum per phi column wanders
    jmax = rho.max(axis=2).argmax(axis=1)
    assert th[jmax].max() - th[jmax].min() > math.radians(100.0)


def test_beta_is_ratio_of_maxima():
    """max p_g / max p_b = 10, with b^2 from the oracle's own conserved variables."""
    geo, prim, bf = _case()
    n1, n2, n3 = geo.n1, geo.n2, geo.n3
    gam = 13.0 / 9.0
    d = O.make_desc(n1, n2, n3, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3, metric=O.METRIC_KS,
                    a=0.9375, gam=gam, bc=(3, 3, 2, 2, 1, 1))
    g = O.Grid(d)
    g.set(prim, bf)
    p, _ = g.get()  # the oracle derives centre B from the faces
    pc = p[:, NG:NG + n3, NG:NG + n2, NG:NG + n1]
    x1 = geo.x1min + (np.arange(n1) + 0.5) * geo.dx1
    x2 = geo.x2min + (np.arange(n2) + 0.5) * geo.dx2
    bsq = np.array([O.state(d, pc[:, k, j, i], x1[i], x2[j])[4]
                    for k in range(n3) for j in range(n2) for i in range(n1)])
    pg = (gam - 1.0) * pc[1]
    assert abs(pg.max() / (0.5 * bsq.max()) - 10.0) < 1e-9 * 10.0


def test_rotation_is_about_the_tilted_axis():
    """The coordinate velocity of a disk cell is perpendicular to both r and the disk normal."""
    geo, prim, _ = _case()
    n1, n2, n3 = geo.n1, geo.n2, geo.n3
    rho = prim[0][NG:NG + n3, NG:NG + n2, NG:NG + n1]
    k, j, i = np.unravel_index(np.argmax(rho), rho.shape)
    r = math.exp(geo.x1min + (i + 0.5) * geo.dx1)
    th = geo.x2min + (j + 0.5) * geo.dx2
    ph = geo.x3min + (k + 0.5) * geo.dx3
    ut2 = prim[3][NG + k, NG + j, NG + i]
    ut3 = prim[4][NG + k, NG + j, NG + i]
    # velocity direction in Cartesian: theta_hat * r ut2 + phi_hat * r sin(th) ut3 (ut1 carries the frame term)
    thhat = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    phhat = np.array([-math.sin(ph), math.cos(ph), 0.0])
    v = thhat * r * ut2 + phhat * r * math.sin(th) * ut3
    tl = math.radians(65.0)
    nvec = np.array([0.0, -math.sin(tl), math.cos(tl)])
    assert abs(v @ nvec) < 1e-12 * np.linalg.norm(v)
    vk = 1.0 / math.sqrt(r)
    assert 0.5 * vk < np.linalg.norm(v) < 2.0 * vk
