"""Pins of the oracle's transmissive polar boundary (Sec. 3.3.1: the grid is
carried across the coordinate singularity; the paper defers the formulas to
its earlier work, so the oracle's rule is a reading: the ghost row j = -1-m
at azimuth k holds the interior row j = m at azimuth k + n3/2, with the
theta components of the velocity and the field negated, and the axis faces
carry no field).

The pins do not restate that rule. They use what it must achieve:

* ghost cells and faces hold the analytic continuation through the axis of
  smooth fields (a point at theta < 0 is the point at -theta, phi + pi):
  scalar fields, and the coordinate components of a uniform Cartesian
  velocity and field, on both poles;
* a state symmetric under the equatorial reflection theta -> pi - theta stays
  symmetric (to round-off: the mirrored cell centres differ by rounding);
* a uniform flow along the axis crosses the pole cells with a truncation
  error that converges (density and internal energy at second order,
  velocity at first) -- a wrong sign or row in the ghost rule leaves an
  error of order one there.

Measured property recorded with them: a uniform flow ACROSS the axis is
not kept to a converging error in the two rows next to the axis (the
reconstructed azimuthal coordinate velocity behaves like 1/sin(theta) and
changes sign across the axis); volume-weighted, the error over the sphere
still converges at first order.
"""
import math

import numpy as np

import oracle as O
from paper_1912_10192_gb300 import workloads as W

NG = O.NG


def sph_desc(n, r0=2.0, r1=4.0, gam=5.0 / 3.0):
    x1a, x1b = math.log(r0), math.log(r1)
    dx = ((x1b - x1a) / n[0], math.pi / n[1], 2 * math.pi / n[2])
    bc = (O.BC_OUTFLOW, O.BC_OUTFLOW, O.BC_POLAR, O.BC_POLAR, O.BC_PERIODIC, O.BC_PERIODIC)
    return O.make_desc(n[0], n[1], n[2], x1a, 0.0, 0.0, *dx, metric=O.METRIC_SPHERICAL, gam=gam, cour=0.5, bc=bc,
                       floors=0)


def cart_to_coord(vec, r, th, ph):
    """Coordinate components (x1 = log r, theta, phi) of a Cartesian vector at (r, th, ph); analytic in th."""
    vx, vy, vz = vec
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    vr = vx * st * cp + vy * st * sp + vz * ct
    vt = vx * ct * cp + vy * ct * sp - vz * st
    vp = -vx * sp + vy * cp
    with np.errstate(divide="ignore", invalid="ignore"):
        return vr / r, vt / r, vp / (r * st)


def scalar_field(r, th, ph):
    """A smooth, non-axisymmetric positive scalar in Cartesian form."""
    x, y, z = r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)
    return 1.0 + 0.2 * np.sin(0.7 * x + 0.3) + 0.1 * np.cos(0.5 * y - 0.4 * z)


def coords(d, i, j, k, face=None):
    """(r, theta, phi) of padded indices; face = None for centres, else 1/2/3 for that face family."""
    x1 = d.x1min + (i - NG + (0.0 if face == 1 else 0.5)) * d.dx1
    x2 = d.x2min + (j - NG + (0.0 if face == 2 else 0.5)) * d.dx2
    x3 = d.x3min + (k - NG + (0.0 if face == 3 else 0.5)) * d.dx3
    return np.exp(x1), x2, x3


def test_ghosts_continue_smooth_fields_through_the_axis():
    n = (6, 8, 12)
    d = sph_desc(n)
    shp = (n[2] + 2 * NG, n[1] + 2 * NG, n[0] + 2 * NG)
    K, J, I = np.meshgrid(*(np.arange(m) for m in shp), indexing="ij")
    v = (0.3, -0.2, 0.25)
    lor = 1.0 / math.sqrt(1.0 - sum(c * c for c in v))
    Bc = (0.4, 0.7, -0.5)

    def fields(face=None):
        r, th, ph = coords(d, I, J, K, face)
        return r, th, ph

    r, th, ph = fields()
    prim = np.zeros((8,) + shp)
    bf = np.zeros((3,) + shp)
    prim[0] = scalar_field(r, th, ph)
    prim[1] = 2.0 * scalar_field(1.3 * r, th, ph + 0.5)     # scaled and rotated about the axis
    u1, u2, u3 = cart_to_coord(v, r, th, ph)
    prim[2], prim[3], prim[4] = lor * u1, lor * u2, lor * u3
    for f in (1, 2, 3):
        rf, thf, phf = fields(f)
        bcomp = cart_to_coord(Bc, rf, thf, phf)[f - 1]
        bf[f - 1] = rf ** 3 * np.abs(np.sin(thf)) * bcomp          # sqrt(-g) B^f at the face centre
    bf[1][:, NG, :] = 0.0
    bf[1][:, NG + n[1], :] = 0.0
    interior = np.zeros(shp, bool)
    interior[NG:NG + n[2], NG:NG + n[1], NG:NG + n[0]] = True
    prim_in = np.where(interior, prim, 0.0)
    bf_in = np.where(interior, bf, 0.0)
    bf_in[0][NG:NG + n[2], NG:NG + n[1], NG + n[0]] = bf[0][NG:NG + n[2], NG:NG + n[1], NG + n[0]]
    bf_in[1][NG:NG + n[2], NG + n[1], NG:NG + n[0]] = 0.0
    bf_in[2][NG + n[2], NG:NG + n[1], NG:NG + n[0]] = bf[2][NG + n[2], NG:NG + n[1], NG:NG + n[0]]
    g = O.Grid(d)
    g.set(prim_in, bf_in)
    P, B = g.get()
    rows = list(range(0, NG)) + list(range(NG + n[1], n[1] + 2 * NG))
    sel = (slice(NG, NG + n[2]), rows, slice(NG, NG + n[0]))
    for v_ in range(5):
        want = prim[v_][sel]
        assert np.abs(P[v_][sel] - want).max() <= 1e-13 * np.abs(want).max(), v_
    # x1- and x3-faces of the ghost rows, and the x2-faces beyond the axis
    for f, frows in ((1, rows), (3, rows), (2, list(range(0, NG)) + list(range(NG + n[1] + 1, n[1] + 2 * NG)))):
        s = (slice(NG, NG + n[2]), frows, slice(NG, NG + n[0]))
        want = bf[f - 1][s]
        assert np.abs(B[f - 1][s] - want).max() <= 1e-13 * np.abs(want).max(), f
    # the axis faces carry no flux
    assert np.all(B[1][:, NG, :] == 0.0) and np.all(B[1][:, NG + n[1], :] == 0.0)
    # centre field of a ghost cell = the face average of its own (ghost) faces over sqrt(-g) there
    for j in rows:
        for k in range(NG, NG + n[2]):
            for i in range(NG, NG + n[0]):
                rr, tt, _ = coords(d, i, j, k)
                gd = rr ** 3 * abs(math.sin(tt))
                b2 = 0.5 * (B[1][k, j, i] + B[1][k, j + 1, i]) / gd if j + 1 < shp[1] else None
                if b2 is not None:
                    assert abs(P[6][k, j, i] - b2) <= 1e-12 * max(1.0, abs(b2)), (j, k, i)


def symmetrise(prim, bf, d):
    """Mirror the northern half of a torus state onto the southern half (equatorial reflection of a
    vector velocity and a pseudo-vector field: utilde^2 odd, Bbar^1 and Bbar^3 odd, Bbar^2 even)."""
    n2 = d.n2
    P, B = prim.copy(), bf.copy()
    for j in range(n2 // 2):
        jm = n2 - 1 - j
        for v in range(8):
            s = -1.0 if v == 3 else 1.0
            P[v][:, NG + jm, :] = s * P[v][:, NG + j, :]
        B[0][:, NG + jm, :] = -B[0][:, NG + j, :]
        B[2][:, NG + jm, :] = -B[2][:, NG + j, :]
    for j in range(n2 // 2):
        B[1][:, NG + n2 - j, :] = B[1][:, NG + j, :]
    return P, B


def test_equatorially_mirrored_torus_stays_mirrored():
    n1, n2, n3 = 24, 16, 8
    geo = W.torus_geometry(n1, n2, n3)
    prim, bf = W.torus_block(geo, seed=5)
    d = O.make_desc(n1, n2, n3, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3, metric=O.METRIC_KS,
                    a=0.9375, gam=13.0 / 9.0, cour=0.8,
                    bc=(O.BC_OUTFLOW_NOINFLOW, O.BC_OUTFLOW_NOINFLOW, O.BC_POLAR, O.BC_POLAR, O.BC_PERIODIC,
                        O.BC_PERIODIC))
    # the perturbed torus with an azimuthal velocity modulated in phi, mirrored about the equator
    prim[4] = prim[4] * (1.0 + 0.05 * np.cos(np.arange(prim.shape[1]) * 2 * math.pi / n3))[:, None, None]
    P0, B0 = symmetrise(prim, bf, d)
    g = O.Grid(d)
    g.set(P0, B0)
    for _ in range(3):
        g.step()
    P, B = g.get()
    core = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
    M, MB = symmetrise(P, B, d)   # the mirror image of the northern half
    for v in range(5):
        a, b = P[v][core], M[v][core]
        assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max(), v
    for f in range(3):
        a, b = B[f][NG:NG + n3 + 1, NG:NG + n2 + 1, NG:NG + n1 + 1], MB[f][NG:NG + n3 + 1, NG:NG + n2 + 1,
                                                                          NG:NG + n1 + 1]
        assert np.abs(a - b).max() <= 1e-11 * max(np.abs(a).max(), 1e-300), f
    # the state is not trivially symmetric because nothing moved: it evolved
    assert np.abs(P[1][core] - P0[1][core]).max() > 1e-8 * np.abs(P0[1][core]).max()


def uniform_flow(n, v, gam=5.0 / 3.0, rho=1.0, p=1.0):
    d = sph_desc(n, gam=gam)
    shp = (n[2] + 2 * NG, n[1] + 2 * NG, n[0] + 2 * NG)
    prim, bf = np.zeros((8,) + shp), np.zeros((3,) + shp)
    x1 = d.x1min + (np.arange(n[0]) + 0.5) * d.dx1
    th = (np.arange(n[1]) + 0.5) * d.dx2
    ph = (np.arange(n[2]) + 0.5) * d.dx3
    PH, TH, X1 = np.meshgrid(ph, th, x1, indexing="ij")
    R = np.exp(X1)
    lor = 1.0 / math.sqrt(1.0 - sum(c * c for c in v))
    s = (slice(NG, NG + n[2]), slice(NG, NG + n[1]), slice(NG, NG + n[0]))
    prim[0][s] = rho
    prim[1][s] = p / (gam - 1.0)
    u = cart_to_coord(v, R, TH, PH)
    for m in range(3):
        prim[2 + m][s] = lor * u[m]
    return d, prim, bf, (R, TH, PH)


def cartesian_state(P, d, rtp):
    R, TH, PH = rtp
    s = (slice(NG, NG + d.n3), slice(NG, NG + d.n2), slice(NG, NG + d.n1))
    u1, u2, u3 = P[2][s] * R, P[3][s] * R, P[4][s] * R * np.sin(TH)
    st, ct, sp, cp = np.sin(TH), np.cos(TH), np.sin(PH), np.cos(PH)
    vx = u1 * st * cp + u2 * ct * cp - u3 * sp
    vy = u1 * st * sp + u2 * ct * sp + u3 * cp
    vz = u1 * ct - u2 * st
    return np.stack([vx, vy, vz, P[0][s], P[1][s]])


def rate_error(n, v):
    """|d state / dt| of one step with a tiny dt (the truncation error of the spatial operator), per
    quantity (Cartesian Gamma v, rho, u_g), radial cells within 3 of the outflow boundaries left out."""
    d, prim, bf, rtp = uniform_flow(n, v)
    g = O.Grid(d)
    g.set(prim, bf)
    p0, _ = g.get()
    dt = 1e-6 * d.dx2
    g.step(dt)
    p1, _ = g.get()
    e = np.abs(cartesian_state(p1, d, rtp) - cartesian_state(p0, d, rtp)) / dt
    return e[..., 3:n[0] - 3], rtp


def test_axial_flow_through_the_pole_converges():
    pole, rest = [], []
    for N in (16, 32, 64):
        e, _ = rate_error((N, N, 4), (0.0, 0.0, 0.6))
        pole.append(e[:, :, :3].mean(axis=(1, 2, 3)))
        rest.append(e[:, :, 3:N // 2].mean(axis=(1, 2, 3)))
    rp = np.log2(pole[1] / pole[2])
    assert rp[2] > 0.85 and rp[3] > 1.8 and rp[4] > 1.8, rp     # v_z first order; rho, u_g second
    assert pole[2][3] < 1e-4 and pole[2][4] < 3e-4, pole[2]
    rr = np.log2(rest[1] / rest[2])
    assert np.all(rr[2:] > 1.6), rr


def test_cross_axis_flow_converges_in_the_volume_norm():
    errs = []
    for N in (8, 16, 32):
        e, (R, TH, _) = rate_error((N, N, 2 * N), (0.3, 0.0, 0.2))
        vol = (R ** 3 * np.sin(TH))[..., 3:N - 3]
        errs.append((e * vol).sum(axis=(1, 2, 3)) / vol.sum())
    rate = np.log2(errs[1] / errs[2])
    assert np.all(rate > 0.9), rate
