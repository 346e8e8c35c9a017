"""Seeded synthetic inputs for the GRMHD block update (host-side numpy).

This module generates initial states only; it holds none of the update's
arithmetic and imports neither the CUDA binding nor the CPU oracle, so both
sides can be fed the same bytes.

* `torus_block`: Fishbone & Moncrief (1976) torus around a Kerr black hole in
  Kerr-Schild coordinates on the log-r spherical grid of Sec. 2.2, with a
  poloidal loop field (A_phi ~ max(rho/rho_max - 0.2, 0) at cell corners,
  face B as its discrete curl) normalised to max p_g / max p_b = beta (the
  same "ratio of maxima" definition the paper uses in Sec. 6.3), and a seeded
  +/- 2% perturbation of u_g inside the torus.
* `random_states`: random primitive states for inversion tests over the
  ranges rho 1e-6..1, u/rho 1e-4..1e2, Lorentz factor 1..50,
  sigma = b^2/rho 0..100, r from just inside the horizon to 100.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014) of
seed XOR global cell id, mapped to [0, 1) with the top 53 bits.
"""
import math

import numpy as np

NG = 3

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """SplitMix64 finaliser of a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform01(seed, ids):
    """xi in [0, 1) for each integer id, from SplitMix64(seed ^ id)."""
    z = splitmix64(np.uint64(seed) ^ np.asarray(ids, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class BlockGeometry:
    """Extents of one block in internal coordinates (x1 = log r, x2 = theta, x3 = phi)."""

    def __init__(self, n1, n2, n3, x1min, x1max, x2min, x2max, x3min, x3max):
        self.n1, self.n2, self.n3 = n1, n2, n3
        self.x1min, self.x2min, self.x3min = x1min, x2min, x3min
        self.dx1 = (x1max - x1min) / n1
        self.dx2 = (x2max - x2min) / n2
        self.dx3 = (x3max - x3min) / n3

    @property
    def padded_shape(self):
        return (self.n3 + 2 * NG, self.n2 + 2 * NG, self.n1 + 2 * NG)


def torus_geometry(n1, n2, n3, rin=1.2, rout=50.0):
    return BlockGeometry(n1, n2, n3, math.log(rin), math.log(rout), 0.0, math.pi, 0.0, 2.0 * math.pi)


# --- Kerr-Schild pieces needed to express the initial state -----------------

def _ks_internal(a, r, th):
    """Non-zero covariant/contravariant KS components in (t, log r, theta, phi)."""
    s2 = np.sin(th) ** 2
    sig = r * r + a * a * np.cos(th) ** 2
    z = 2.0 * r / sig
    gcov = {
        (0, 0): -(1.0 - z), (0, 1): z * r, (0, 3): -z * a * s2, (1, 1): (1.0 + z) * r * r,
        (1, 3): -a * s2 * (1.0 + z) * r, (2, 2): sig, (3, 3): s2 * (sig + a * a * s2 * (1.0 + z)),
    }
    for (m, n) in list(gcov):
        if m != n:
            gcov[(n, m)] = gcov[(m, n)]
    gtt_con = -(1.0 + z)
    gt1_con = z / r
    gdet = r * sig * np.sin(th)
    return gcov, gtt_con, gt1_con, gdet


def _fm_lnh(a, r, th, ell):
    """Fishbone-Moncrief log-enthalpy (constant u^t u_phi = ell) in BL, up to a constant."""
    s2 = np.sin(th) ** 2
    sig = r * r + a * a * np.cos(th) ** 2
    dlt = r * r - 2.0 * r + a * a
    A = (r * r + a * a) ** 2 - dlt * a * a * s2
    q = np.sqrt(1.0 + 4.0 * ell * ell * sig * sig * dlt / (A * A * s2))
    return 0.5 * np.log((1.0 + q) / (sig * dlt / A)) - 0.5 * q - 2.0 * a * r * ell / A


def fm_ell(a, rmax):
    """u^t u_phi of the prograde circular equatorial geodesic at rmax (pressure maximum)."""
    sr = math.sqrt(rmax)
    return ((rmax ** 1.5 + a) * (rmax * rmax - 2.0 * a * sr + a * a)
            / (rmax ** 1.5 * (rmax ** 1.5 - 3.0 * sr + 2.0 * a)))


def _fm_velocity_bl(a, r, th, ell):
    """(u^t, u^phi) in Boyer-Lindquist for the FM torus."""
    s2 = np.sin(th) ** 2
    sig = r * r + a * a * np.cos(th) ** 2
    dlt = r * r - 2.0 * r + a * a
    A = (r * r + a * a) ** 2 - dlt * a * a * s2
    gtt = -A / (sig * dlt)
    gtp = -2.0 * a * r / (sig * dlt)
    gpp = (dlt - a * a * s2) / (sig * dlt * s2)
    K = gtp * gtp - gtt * gpp
    uphi_cov = np.sqrt((gtt + np.sqrt(gtt * gtt + 4.0 * K * ell * ell)) / (2.0 * K))
    ut_cov = (ell - gtp * uphi_cov ** 2) / (gtt * uphi_cov)
    ut = gtt * ut_cov + gtp * uphi_cov
    uphi = gtp * ut_cov + gpp * uphi_cov
    return ut, uphi


def _bsq(a, r, th, prim_u, Bcon):
    """b^2 for utilde^i = prim_u[0..2] and centre B^i = Bcon[0..2] (broadcast arrays)."""
    gcov, gtt_con, gt1_con, _ = _ks_internal(a, r, th)
    alpha = 1.0 / np.sqrt(-gtt_con)
    qsq = sum(gcov[(i + 1, j + 1)] * prim_u[i] * prim_u[j]
              for i in range(3) for j in range(3) if (i + 1, j + 1) in gcov)
    gamma = np.sqrt(1.0 + qsq)
    ucon = [gamma / alpha, prim_u[0] - gamma * alpha * gt1_con, prim_u[1], prim_u[2]]
    ucov = [sum(gcov[(m, n)] * ucon[n] for n in range(4) if (m, n) in gcov) for m in range(4)]
    bt = sum(Bcon[i] * ucov[i + 1] for i in range(3))
    bcon = [bt] + [(Bcon[i] + bt * ucon[i + 1]) / ucon[0] for i in range(3)]
    return sum(gcov[(m, n)] * bcon[m] * bcon[n] for m in range(4) for n in range(4) if (m, n) in gcov)


def torus_block(geo, a=0.9375, gam=13.0 / 9.0, rin=6.0, rmax=12.0, beta=100.0, pert=0.02, seed=1912,
                kappa=1.0e-3):
    """Padded primitive (8, n3p, n2p, n1p) and face-B (3, ...) arrays of the magnetised FM torus.

    Ghost zones are left at zero: each side fills them with its own boundary
    conditions. Centre B^i (prim slots 5..7) is left at zero too: it is a
    function of the face field, computed by each side.
    """
    n1, n2, n3 = geo.n1, geo.n2, geo.n3
    shp = geo.padded_shape
    prim = np.zeros((8,) + shp)
    bface = np.zeros((3,) + shp)
    ell = fm_ell(a, rmax)
    lnh_in = _fm_lnh(a, rin, 0.5 * math.pi, ell)

    i = np.arange(n1)
    j = np.arange(n2)
    x1 = geo.x1min + (i + 0.5) * geo.dx1
    x2 = geo.x2min + (j + 0.5) * geo.dx2
    R, TH = np.meshgrid(np.exp(x1), x2, indexing="xy")  # (n2, n1)
    rplus = 1.0 + math.sqrt(1.0 - a * a)

    def torus_rho_u(r, th):
        with np.errstate(invalid="ignore", divide="ignore"):
            lnh = np.where(r > rplus * 1.0001, _fm_lnh(a, r, th, ell) - lnh_in, -1.0)
        inside = (r >= rin) & (lnh > 0.0)
        hm1 = np.where(inside, np.exp(np.where(inside, lnh, 0.0)) - 1.0, 0.0)
        rho = np.where(inside, (hm1 * (gam - 1.0) / (kappa * gam)) ** (1.0 / (gam - 1.0)), 0.0)
        u = kappa * rho ** gam / (gam - 1.0)
        return rho, u, inside

    rho_t, u_t, inside = torus_rho_u(R, TH)
    rhomax = rho_t.max()
    rho_t /= rhomax
    u_t /= rhomax

    # velocities (Kerr-Schild, internal coordinates)
    ut_bl, uphi_bl = _fm_velocity_bl(a, np.where(inside, R, 20.0), np.where(inside, TH, 1.5), ell)
    gcov, gtt_con, gt1_con, _ = _ks_internal(a, R, TH)
    alpha = 1.0 / np.sqrt(-gtt_con)
    gamma_n = alpha * ut_bl  # u^t_KS = u^t_BL when u^r = 0
    ut1 = np.where(inside, gamma_n * alpha * gt1_con, 0.0)
    ut3 = np.where(inside, uphi_bl, 0.0)

    rho_flr = 1.0e-7 / R ** 2
    u_flr = 1.0e-9 * R ** (-10.0 / 3.0)
    rho = np.maximum(rho_t, rho_flr)
    u = np.maximum(u_t, u_flr)

    # perturbation inside the torus, keyed by the global (block-local here) cell id
    kk, jj, ii = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    ids = (ii + n1 * (jj + n2 * kk)).astype(np.uint64)
    xi = uniform01(seed, ids)
    u3 = np.broadcast_to(u, (n3, n2, n1)).copy()
    u3 = np.where(np.broadcast_to(inside, (n3, n2, n1)), u3 * (1.0 + pert * (2.0 * xi - 1.0)), u3)

    s = (slice(None), slice(NG, NG + n2), slice(NG, NG + n1))
    sk = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
    prim[0][s] = rho
    prim[1][sk] = u3
    prim[2][s] = ut1
    prim[3][s] = 0.0
    prim[4][s] = ut3

    # loop field: A_phi at cell corners (i-1/2, j-1/2)
    xc1 = geo.x1min + np.arange(n1 + 1) * geo.dx1
    xc2 = geo.x2min + np.arange(n2 + 1) * geo.dx2
    RC, THC = np.meshgrid(np.exp(xc1), xc2, indexing="xy")  # (n2+1, n1+1)
    rho_c, _, _ = torus_rho_u(RC, THC)
    Aphi = np.maximum(rho_c / rhomax - 0.2, 0.0)
    b1 = (Aphi[1:, :] - Aphi[:-1, :]) / geo.dx2        # (n2, n1+1): faces i = 0..n1
    b2 = -(Aphi[:, 1:] - Aphi[:, :-1]) / geo.dx1       # (n2+1, n1): faces j = 0..n2
    # axis faces carry no flux area
    b2[0, :] = 0.0 if geo.x2min == 0.0 else b2[0, :]
    if abs(geo.x2min + n2 * geo.dx2 - math.pi) < 1e-12:
        b2[-1, :] = 0.0

    # normalise to beta = max p_g / max p_b using centre B = <Bbar>/sqrt(-g)
    _, _, _, gdet = _ks_internal(a, R, TH)
    Bc1 = 0.5 * (b1[:, :-1] + b1[:, 1:]) / gdet
    Bc2 = 0.5 * (b2[:-1, :] + b2[1:, :]) / gdet
    bsq = _bsq(a, R, TH, (ut1, np.zeros_like(ut1), ut3), (Bc1, Bc2, np.zeros_like(Bc1)))
    pg_max = ((gam - 1.0) * u3).max()
    pb_max = 0.5 * bsq.max()
    if pb_max > 0.0 and beta > 0.0:
        fac = math.sqrt(pg_max / (beta * pb_max))
    else:
        fac = 0.0
    for k in range(n3):
        bface[0, NG + k, NG:NG + n2, NG:NG + n1 + 1] = fac * b1
        bface[1, NG + k, NG:NG + n2 + 1, NG:NG + n1] = fac * b2
    return prim, bface


def random_states(n, seed, a=0.9375, rho_range=(1e-6, 1.0), urho_range=(1e-4, 1e2), lorentz_range=(1.0, 50.0),
                  sigma_range=(0.0, 100.0), rmax=100.0):
    """Random primitive states and positions for inversion tests.

    Returns prim (n, 8) with centre B^i in slots 5..7, and x1 = log r, x2 = theta.
    Directions of utilde^i and B^i are isotropic in the local coordinate basis
    normalised by g_ij.
    """
    ids = np.arange(n, dtype=np.uint64) * np.uint64(16)
    xi = [uniform01(seed, ids + np.uint64(m)) for m in range(12)]
    rplus = 1.0 + math.sqrt(1.0 - a * a)
    r = np.exp(math.log(0.9 * rplus) + xi[0] * (math.log(rmax) - math.log(0.9 * rplus)))
    cth = 2.0 * xi[1] - 1.0
    cth = np.clip(cth, -math.sqrt(1.0 - 1e-6), math.sqrt(1.0 - 1e-6))
    th = np.arccos(cth)
    rho = np.exp(np.log(rho_range[0]) + xi[2] * (np.log(rho_range[1]) - np.log(rho_range[0])))
    u = rho * np.exp(np.log(urho_range[0]) + xi[3] * (np.log(urho_range[1]) - np.log(urho_range[0])))
    lor = np.exp(np.log(lorentz_range[0]) + xi[4] * (np.log(lorentz_range[1]) - np.log(lorentz_range[0])))
    sigma = sigma_range[0] + xi[5] * (sigma_range[1] - sigma_range[0])

    def iso(x, y):
        z = 2.0 * x - 1.0
        ph = 2.0 * math.pi * y
        s = np.sqrt(1.0 - z * z)
        return np.stack([s * np.cos(ph), s * np.sin(ph), z])

    gcov, _, _, _ = _ks_internal(a, r, th)

    def gnorm(v):
        return np.sqrt(sum(gcov[(i + 1, j + 1)] * v[i] * v[j]
                           for i in range(3) for j in range(3) if (i + 1, j + 1) in gcov))

    nu = iso(xi[6], xi[7])
    nu = nu / gnorm(nu)
    utl = np.sqrt(lor * lor - 1.0) * nu
    nb = iso(xi[8], xi[9])
    nb = nb / gnorm(nb)
    b2unit = _bsq(a, r, th, utl, nb)
    scale = np.sqrt(sigma * rho / b2unit)
    B = nb * scale
    prim = np.stack([rho, u, utl[0], utl[1], utl[2], B[0], B[1], B[2]], axis=1)
    return prim, np.log(r), th


# --- multi-block inputs ------------------------------------------------------
#
# A block is described by a plain dict: n1, n2, n3, x1min, x2min, x3min, dx1,
# dx2, dx3, bc (6 ints: 0 outflow, 1 periodic, 2 polar, 3 no-inflow outflow,
# 4 neighbouring block) and lat (local time-step level).

BC_BLOCK = 4


def _edges(lo, h, n):
    return lo + np.arange(n + 1) * h


def _centres(lo, h, n):
    return lo + (np.arange(n) + 0.5) * h


def flat_box_tree(base=(2, 2, 2), n=8, refine=((0, 0, 0),), lat_coarse=1, lat_fine=0, L=1.0):
    """Periodic unit box of base[0] x base[1] x base[2] blocks of n^3 cells (n
    may be a triple); the listed base blocks are split into 8 children with
    the same cell counts (2x finer)."""
    blocks = []
    nn = (n, n, n) if isinstance(n, int) else tuple(n)
    hb = [L / base[d] for d in range(3)]
    for kb in range(base[2]):
        for jb in range(base[1]):
            for ib in range(base[0]):
                lo = (ib * hb[0], jb * hb[1], kb * hb[2])
                if (ib, jb, kb) in refine:
                    for kc in range(2):
                        for jc in range(2):
                            for ic in range(2):
                                blocks.append(dict(n1=nn[0], n2=nn[1], n3=nn[2], x1min=lo[0] + ic * hb[0] / 2,
                                                   x2min=lo[1] + jc * hb[1] / 2, x3min=lo[2] + kc * hb[2] / 2,
                                                   dx1=hb[0] / (2 * nn[0]), dx2=hb[1] / (2 * nn[1]),
                                                   dx3=hb[2] / (2 * nn[2]), bc=[1, 1, 1, 1, 1, 1], lat=lat_fine))
                else:
                    blocks.append(dict(n1=nn[0], n2=nn[1], n3=nn[2], x1min=lo[0], x2min=lo[1], x3min=lo[2],
                                       dx1=hb[0] / nn[0], dx2=hb[1] / nn[1], dx3=hb[2] / nn[2],
                                       bc=[1, 1, 1, 1, 1, 1], lat=lat_coarse))
    _mark_block_faces(blocks, periodic=(True, True, True))
    return blocks


def split6(b, axis_low=True):
    """The 6-way split of a block (Sec. 3.3.1) with its 'axis' at the lower (axis_low) or upper x2 side:
    the x2 half at the axis gives 2 children (halved in x1 and x2, the parent's x3 extent and cells),
    the other half 4 children halved in all three directions; every child keeps the parent's cell
    counts. Returns the 6 block dicts (bc copied, lat kept)."""
    h = (b["n1"] * b["dx1"] / 2, b["n2"] * b["dx2"] / 2, b["n3"] * b["dx3"] / 2)
    out = []
    for jc in range(2):
        for ic in range(2):
            lo = (b["x1min"] + ic * h[0], b["x2min"] + jc * h[1])
            if (jc == 0) == axis_low:
                out.append(dict(b, x1min=lo[0], x2min=lo[1], x3min=b["x3min"], dx1=b["dx1"] / 2,
                                dx2=b["dx2"] / 2, dx3=b["dx3"], bc=list(b["bc"])))
            else:
                for kc in range(2):
                    out.append(dict(b, x1min=lo[0], x2min=lo[1], x3min=b["x3min"] + kc * h[2], dx1=b["dx1"] / 2,
                                    dx2=b["dx2"] / 2, dx3=b["dx3"] / 2, bc=list(b["bc"])))
    return out


def flat_box_tree6(base=(2, 2, 2), n=6, split=((0, 0, 0),), refine=(), L=1.0, lat=0):
    """Periodic flat box of base blocks of n^3 cells; the base blocks listed in `split` are split 6-way
    (split6, the axis on their lower x2 side), those in `refine` into 8 octants."""
    blocks = []
    nn = (n, n, n) if isinstance(n, int) else tuple(n)
    hb = [L / base[d] for d in range(3)]
    for kb in range(base[2]):
        for jb in range(base[1]):
            for ib in range(base[0]):
                b = dict(n1=nn[0], n2=nn[1], n3=nn[2], x1min=ib * hb[0], x2min=jb * hb[1], x3min=kb * hb[2],
                         dx1=hb[0] / nn[0], dx2=hb[1] / nn[1], dx3=hb[2] / nn[2], bc=[1] * 6, lat=lat)
                if (ib, jb, kb) in split:
                    blocks.extend(split6(b))
                elif (ib, jb, kb) in refine:
                    for kc in range(2):
                        for jc in range(2):
                            for ic in range(2):
                                blocks.append(dict(b, x1min=b["x1min"] + ic * hb[0] / 2,
                                                   x2min=b["x2min"] + jc * hb[1] / 2,
                                                   x3min=b["x3min"] + kc * hb[2] / 2, dx1=b["dx1"] / 2,
                                                   dx2=b["dx2"] / 2, dx3=b["dx3"] / 2, bc=[1] * 6))
                else:
                    blocks.append(b)
    _mark_block_faces(blocks, periodic=(True, True, True))
    return blocks


def _mark_block_faces(blocks, periodic):
    """Faces interior to the domain get BC_BLOCK; faces on the domain boundary
    keep their bc (periodic ones too: the neighbour across the period is
    found by position)."""
    lo = [min(b["x%dmin" % (d + 1)] for b in blocks) for d in range(3)]
    hi = [max(b["x%dmin" % (d + 1)] + b["n%d" % (d + 1)] * b["dx%d" % (d + 1)] for b in blocks) for d in range(3)]
    for b in blocks:
        for d in range(3):
            blo = b["x%dmin" % (d + 1)]
            bhi = blo + b["n%d" % (d + 1)] * b["dx%d" % (d + 1)]
            tol = 1e-9 * (hi[d] - lo[d])
            if blo > lo[d] + tol:
                b["bc"][2 * d] = BC_BLOCK
            if bhi < hi[d] - tol:
                b["bc"][2 * d + 1] = BC_BLOCK


def flat_box_state(blocks, gam=5.0 / 3.0, amp=0.1, bamp=0.05, L=1.0):
    """Smooth periodic state on each block: padded prim and face-B arrays.
    Face B is the discrete curl of an edge vector potential whose components
    do not vary along their own direction (A1(y,z), A2(z,x), A3(x,y)), so the
    flux of a coarse face is exactly the sum of its finer faces'."""
    tp = 2.0 * math.pi / L
    A1 = lambda y, z: bamp * np.cos(tp * y + tp * z) / tp
    A2 = lambda z, x: bamp * np.sin(tp * z) * np.cos(tp * x) / tp
    A3 = lambda x, y: bamp * np.sin(tp * x) * np.sin(tp * y) / tp
    out = []
    for b in blocks:
        n1, n2, n3 = b["n1"], b["n2"], b["n3"]
        x = _centres(b["x1min"], b["dx1"], n1)
        y = _centres(b["x2min"], b["dx2"], n2)
        z = _centres(b["x3min"], b["dx3"], n3)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        shp = (n3 + 2 * NG, n2 + 2 * NG, n1 + 2 * NG)
        prim = np.zeros((8,) + shp)
        bf = np.zeros((3,) + shp)
        s = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
        prim[0][s] = 1.0 + amp * np.sin(tp * X + 1.0) * np.cos(tp * Y)
        prim[1][s] = 1.0 + amp * np.cos(tp * Z + 2 * tp * X)
        prim[2][s] = 0.3 + amp * np.sin(tp * Y)
        prim[3][s] = -0.2 + amp * np.sin(tp * (X + Z))
        prim[4][s] = 0.1 + amp * np.cos(tp * X)
        xe = _edges(b["x1min"], b["dx1"], n1)
        ye = _edges(b["x2min"], b["dx2"], n2)
        ze = _edges(b["x3min"], b["dx3"], n3)
        # Bbar1 on x-faces (xe[i], y_c, z_c), i = 0..n1: dA3/dy - dA2/dz
        Zc, Yc, Xe = np.meshgrid(z, y, xe, indexing="ij")
        b1 = ((A3(Xe, Yc + 0.5 * b["dx2"]) - A3(Xe, Yc - 0.5 * b["dx2"])) / b["dx2"]
              - (A2(Zc + 0.5 * b["dx3"], Xe) - A2(Zc - 0.5 * b["dx3"], Xe)) / b["dx3"])
        Zc, Ye, Xc = np.meshgrid(z, ye, x, indexing="ij")
        b2 = ((A1(Ye, Zc + 0.5 * b["dx3"]) - A1(Ye, Zc - 0.5 * b["dx3"])) / b["dx3"]
              - (A3(Xc + 0.5 * b["dx1"], Ye) - A3(Xc - 0.5 * b["dx1"], Ye)) / b["dx1"])
        Ze, Yc, Xc = np.meshgrid(ze, y, x, indexing="ij")
        b3 = ((A2(Ze, Xc + 0.5 * b["dx1"]) - A2(Ze, Xc - 0.5 * b["dx1"])) / b["dx1"]
              - (A1(Yc + 0.5 * b["dx2"], Ze) - A1(Yc - 0.5 * b["dx2"], Ze)) / b["dx2"])
        bf[0][NG:NG + n3, NG:NG + n2, NG:NG + n1 + 1] = b1
        bf[1][NG:NG + n3, NG:NG + n2 + 1, NG:NG + n1] = b2
        bf[2][NG:NG + n3 + 1, NG:NG + n2, NG:NG + n1] = b3
        out.append((prim, bf))
    return out


def torus_tree(nb=(2, 2, 2), n=(8, 8, 8), refine=(), rin=1.2, rout=50.0, lat_base=0, lat_refined=0):
    """Spherical-polar Kerr-Schild domain (log r in [log rin, log rout], theta
    in [0, pi], phi in [0, 2 pi)) of nb base blocks of n cells; the listed base
    blocks (ib, jb, kb) are split into 8 children with the same cell counts."""
    x1a, x1b = math.log(rin), math.log(rout)
    ext = (x1b - x1a, math.pi, 2.0 * math.pi)
    lo0 = (x1a, 0.0, 0.0)
    hb = [ext[d] / nb[d] for d in range(3)]
    blocks = []
    for kb in range(nb[2]):
        for jb in range(nb[1]):
            for ib in range(nb[0]):
                lo = (lo0[0] + ib * hb[0], lo0[1] + jb * hb[1], lo0[2] + kb * hb[2])
                if (ib, jb, kb) in refine:
                    for kc in range(2):
                        for jc in range(2):
                            for ic in range(2):
                                blocks.append(dict(n1=n[0], n2=n[1], n3=n[2], x1min=lo[0] + ic * hb[0] / 2,
                                                   x2min=lo[1] + jc * hb[1] / 2, x3min=lo[2] + kc * hb[2] / 2,
                                                   dx1=hb[0] / (2 * n[0]), dx2=hb[1] / (2 * n[1]),
                                                   dx3=hb[2] / (2 * n[2]), bc=[3, 3, 2, 2, 1, 1], lat=lat_refined))
                else:
                    blocks.append(dict(n1=n[0], n2=n[1], n3=n[2], x1min=lo[0], x2min=lo[1], x3min=lo[2],
                                       dx1=hb[0] / n[0], dx2=hb[1] / n[1], dx3=hb[2] / n[2], bc=[3, 3, 2, 2, 1, 1],
                                       lat=lat_base))
    _mark_block_faces(blocks, periodic=(False, False, True))
    return blocks


def torus_blocks(blocks, a=0.9375, gam=13.0 / 9.0, rin=6.0, rmax=12.0, beta=100.0, pert=0.02, seed=3,
                 kappa=1.0e-3):
    """The magnetised FM torus of `torus_block` on a list of blocks: rho_max = 1
    and max p_g / max p_b = beta over all blocks; A_phi is the same function of
    position everywhere, so the face field is consistent across blocks.
    Perturbation ids: block index * 2^40 + local cell id."""
    ell = fm_ell(a, rmax)
    lnh_in = _fm_lnh(a, rin, 0.5 * math.pi, ell)
    rplus = 1.0 + math.sqrt(1.0 - a * a)

    def torus_rho_u(r, th):
        with np.errstate(invalid="ignore", divide="ignore"):
            lnh = np.where(r > rplus * 1.0001, _fm_lnh(a, r, th, ell) - lnh_in, -1.0)
        inside = (r >= rin) & (lnh > 0.0)
        hm1 = np.where(inside, np.exp(np.where(inside, lnh, 0.0)) - 1.0, 0.0)
        rho = np.where(inside, (hm1 * (gam - 1.0) / (kappa * gam)) ** (1.0 / (gam - 1.0)), 0.0)
        return rho, inside

    rhomax = 0.0
    for b in blocks:
        R, TH = np.meshgrid(np.exp(_centres(b["x1min"], b["dx1"], b["n1"])), _centres(b["x2min"], b["dx2"], b["n2"]),
                            indexing="xy")
        rhomax = max(rhomax, torus_rho_u(R, TH)[0].max())
    out, pg_max, pb_max = [], 0.0, 0.0
    for bi, b in enumerate(blocks):
        n1, n2, n3 = b["n1"], b["n2"], b["n3"]
        R, TH = np.meshgrid(np.exp(_centres(b["x1min"], b["dx1"], n1)), _centres(b["x2min"], b["dx2"], n2),
                            indexing="xy")
        rho_t, inside = torus_rho_u(R, TH)
        rho_t = rho_t / rhomax
        u_t = kappa * (rho_t * rhomax) ** gam / (gam - 1.0) / rhomax
        ut_bl, uphi_bl = _fm_velocity_bl(a, np.where(inside, R, 20.0), np.where(inside, TH, 1.5), ell)
        gcov, gtt_con, gt1_con, gdet = _ks_internal(a, R, TH)
        alpha = 1.0 / np.sqrt(-gtt_con)
        ut1 = np.where(inside, alpha * ut_bl * alpha * gt1_con, 0.0)
        ut3 = np.where(inside, uphi_bl, 0.0)
        rho = np.maximum(rho_t, 1.0e-7 / R ** 2)
        u = np.maximum(u_t, 1.0e-9 * R ** (-10.0 / 3.0))
        kk, jj, ii = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
        ids = (ii + n1 * (jj + n2 * kk)).astype(np.uint64) + np.uint64(bi) * np.uint64(1 << 40)
        xi = uniform01(seed, ids)
        u3 = np.broadcast_to(u, (n3, n2, n1)).copy()
        u3 = np.where(np.broadcast_to(inside, (n3, n2, n1)), u3 * (1.0 + pert * (2.0 * xi - 1.0)), u3)
        shp = (n3 + 2 * NG, n2 + 2 * NG, n1 + 2 * NG)
        prim = np.zeros((8,) + shp)
        bf = np.zeros((3,) + shp)
        s2 = (slice(None), slice(NG, NG + n2), slice(NG, NG + n1))
        s3 = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
        prim[0][s2] = rho
        prim[1][s3] = u3
        prim[2][s2] = ut1
        prim[4][s2] = ut3
        # loop field at corners (x1 faces x x2 faces), same for every phi
        RC, THC = np.meshgrid(np.exp(_edges(b["x1min"], b["dx1"], n1)), _edges(b["x2min"], b["dx2"], n2),
                              indexing="xy")
        rho_c, _ = torus_rho_u(RC, THC)
        Aphi = np.maximum(rho_c / rhomax - 0.2, 0.0)
        b1 = (Aphi[1:, :] - Aphi[:-1, :]) / b["dx2"]
        b2 = -(Aphi[:, 1:] - Aphi[:, :-1]) / b["dx1"]
        if abs(b["x2min"]) < 1e-12:
            b2[0, :] = 0.0
        if abs(b["x2min"] + n2 * b["dx2"] - math.pi) < 1e-12:
            b2[-1, :] = 0.0
        Bc1 = 0.5 * (b1[:, :-1] + b1[:, 1:]) / gdet
        Bc2 = 0.5 * (b2[:-1, :] + b2[1:, :]) / gdet
        bsq = _bsq(a, R, TH, (ut1, np.zeros_like(ut1), ut3), (Bc1, Bc2, np.zeros_like(Bc1)))
        pg_max = max(pg_max, ((gam - 1.0) * u3).max())
        pb_max = max(pb_max, 0.5 * bsq.max())
        for k in range(n3):
            bf[0, NG + k, NG:NG + n2, NG:NG + n1 + 1] = b1
            bf[1, NG + k, NG:NG + n2 + 1, NG:NG + n1] = b2
        out.append((prim, bf))
    fac = math.sqrt(pg_max / (beta * pb_max)) if (pb_max > 0.0 and beta > 0.0) else 0.0
    for prim, bf in out:
        bf *= fac
    return out


def _box(b):
    lo = [b["x1min"], b["x2min"], b["x3min"]]
    hi = [lo[d] + b["n%d" % (d + 1)] * b["dx%d" % (d + 1)] for d in range(3)]
    return lo, hi


def _touch(a, b, period3):
    """blocks a and b share a face, an edge or a corner (phi periodic)"""
    la, ha = _box(a)
    lb, hb = _box(b)
    for d in range(3):
        tol = 1e-9 * max(ha[d] - la[d], hb[d] - lb[d])
        if d == 2 and period3:
            ok = any(la[d] <= hb[d] + s + tol and lb[d] + s <= ha[d] + tol for s in (-period3, 0.0, period3))
        else:
            ok = la[d] <= hb[d] + tol and lb[d] <= ha[d] + tol
        if not ok:
            return False
    return True


def smr_row_widths(blocks, smr):
    """Internal SMR (Sec. 3.3.2): the group width in x3 of every row of every block (1 where not
    grouped), by the rows and phi ranges of the coarsest polar blocks: a row at distance jp (in the
    coarsest polar blocks' rows) from a polar face is grouped 2^n wide, n the largest level with
    jp < 2^(smr - n); a block with 2^l2 times finer x2 cells and 2^l3 times finer x3 cells groups
    2^l3 times as many of its own cells. Returns one array of n2 widths per block."""
    polar = [b for b in blocks if 2 in (b["bc"][2], b["bc"][3])]
    out = []
    for b in blocks:
        w = np.ones(b["n2"], dtype=int)
        if smr > 0 and b in polar:
            l2 = int(round(math.log2(max(p["dx2"] for p in polar) / b["dx2"])))
            l3 = int(round(math.log2(max(p["dx3"] for p in polar) / b["dx3"])))
            for j in range(b["n2"]):
                jp = 1 << 30
                if b["bc"][2] == 2:
                    jp = j
                if b["bc"][3] == 2:
                    jp = min(jp, b["n2"] - 1 - j)
                for lev in range(smr, 0, -1):
                    if (jp >> l2) < 2 ** (smr - lev):
                        w[j] = 2 ** lev * 2 ** l3
                        break
        out.append(w)
    return out


def assign_lat_levels(blocks, lmax=3, period3=2.0 * math.pi, smr=0):
    """LAT levels from the light-crossing time of each block's smallest cell
    in Kerr-Schild internal coordinates, dt_b ~ min over cells of
    1 / (1/(r dx1) + 1/(r dx2) + 1/(r sin(theta) dx3 w)) (a state-independent
    stand-in for the CFL condition, Sec. 3.4; w the row's internal-SMR group
    width, 1 without), level = min(lmax, floor(log2(dt_b / min dt))); then
    smoothed so that blocks that touch differ by at most one level and a
    spatially finer block is never on a coarser time level than a block it
    touches."""
    dts = []
    widths = smr_row_widths(blocks, smr)
    for b, w in zip(blocks, widths):
        x1 = _centres(b["x1min"], b["dx1"], b["n1"])
        x2 = _centres(b["x2min"], b["dx2"], b["n2"])
        R, TH = np.meshgrid(np.exp(x1), x2, indexing="ij")
        inv = 1.0 / (R * b["dx1"]) + 1.0 / (R * b["dx2"]) + 1.0 / (R * np.abs(np.sin(TH)) * b["dx3"] * w[None, :])
        dts.append(float((1.0 / inv).min()))
    dmin = min(dts)
    lat = [min(lmax, int(math.floor(math.log2(d / dmin) + 1e-9))) for d in dts]
    nbh = [[j for j in range(len(blocks)) if j != i and _touch(blocks[i], blocks[j], period3)]
           for i in range(len(blocks))]
    vol = [b["dx1"] * b["dx2"] * b["dx3"] for b in blocks]
    changed = True
    while changed:
        changed = False
        for i in range(len(blocks)):
            for j in nbh[i]:
                if lat[i] > lat[j] + 1:
                    lat[i] = lat[j] + 1
                    changed = True
                if vol[i] < vol[j] * (1 - 1e-9) and lat[i] > lat[j]:
                    lat[i] = lat[j]
                    changed = True
    for b, L in zip(blocks, lat):
        b["lat"] = L
    return blocks


def polar_smr_tree(rin, rout, nb=(8, 4, 4), n=32, refine_ib=range(2, 6), lmax=3):
    """Blocks over r in [rin, rout] (log), theta in [0, pi], phi in [0, 2 pi): a base of
    nb blocks, n^3 cells near the equator and n x n x n/2 within pi/nb[1] of the poles (phi
    derefined, external SMR, Sec. 3.3.1); base blocks at the radial indices refine_ib are refined:
    equatorial ones into 8 octants of n^3 cells, polar ones 6-way (Sec. 3.3.1: 4 octants refined in
    every direction and the 2 children on the axis refined in r and theta only), all n x n x n/2.
    LAT levels from assign_lat_levels (at most lmax)."""
    x1a, x1b = math.log(rin), math.log(rout)
    hb = ((x1b - x1a) / nb[0], math.pi / nb[1], 2.0 * math.pi / nb[2])
    blocks = []

    def add(lo, ext, cells):
        blocks.append(dict(n1=cells[0], n2=cells[1], n3=cells[2], x1min=lo[0], x2min=lo[1], x3min=lo[2],
                           dx1=ext[0] / cells[0], dx2=ext[1] / cells[1], dx3=ext[2] / cells[2],
                           bc=[3, 3, 2, 2, 1, 1], lat=0))

    for kb in range(nb[2]):
        for jb in range(nb[1]):
            for ib in range(nb[0]):
                lo = (x1a + ib * hb[0], jb * hb[1], kb * hb[2])
                polar = jb in (0, nb[1] - 1)
                cells = (n, n, n // 2) if polar else (n, n, n)
                if ib not in refine_ib:
                    add(lo, hb, cells)
                    continue
                half = (hb[0] / 2, hb[1] / 2, hb[2] / 2)
                for jc in range(2):
                    for ic in range(2):
                        clo = (lo[0] + ic * half[0], lo[1] + jc * half[1])
                        axis = polar and ((jb == 0 and jc == 0) or (jb == nb[1] - 1 and jc == 1))
                        if axis:  # keeps the parent's phi cells and extent
                            add((clo[0], clo[1], lo[2]), (half[0], half[1], hb[2]), (n, n, n // 2))
                        else:
                            for kc in range(2):
                                add((clo[0], clo[1], lo[2] + kc * half[2]), half, cells)
    _mark_block_faces(blocks, periodic=(False, False, True))
    return assign_lat_levels(blocks, lmax=lmax)


def c3_blocks(nb=(8, 4, 4), n=32, rin=1.2, rout=50.0, disk=None, level2=None, polar_split=range(2, 6),
              polar_cells=None, axis_cells=None, far_cells=None):
    """Blocks of a two-level refined torus grid over r in [rin, rout] (log), theta in [0, pi],
    phi in [0, 2 pi): a base of nb blocks of n^3 cells; base rows next to the poles (theta index 0
    and nb[1] - 1) derefined in phi (external SMR, Sec. 3.3.1: polar_cells, default n x n x n/2);
    the base blocks (ib, jb) of `disk` (all phi) split into 8 octants of n^3 cells (level 1); the
    level-1 blocks (i1, j1) of `level2` (global level-1 indices, all phi) split again (level 2);
    the polar base blocks at the radial indices `polar_split` split 6-way (Sec. 3.3.1: the two
    children on the axis keep the parent's phi resolution and halve r and theta, the four others
    halve all three; default cell counts: both n x n x n/2, i.e. axis_cells and far_cells).
    Each block carries "level" (spatial refinement level) and "group" (for the histogram)."""
    if disk is None:
        disk = {(ib, jb) for ib in (3, 4) for jb in (1, 2)}
    if level2 is None:
        level2 = {(8, j1) for j1 in (3, 4)}
    polar_cells = polar_cells or (n, n, n // 2)
    axis_cells = axis_cells or (n, n, n // 2)
    far_cells = far_cells or (n, n, n // 2)
    x1a, x1b = math.log(rin), math.log(rout)
    hb = ((x1b - x1a) / nb[0], math.pi / nb[1], 2.0 * math.pi / nb[2])
    blocks = []

    def add(lo, ext, cells, level, group):
        blocks.append(dict(n1=cells[0], n2=cells[1], n3=cells[2], x1min=lo[0], x2min=lo[1], x3min=lo[2],
                           dx1=ext[0] / cells[0], dx2=ext[1] / cells[1], dx3=ext[2] / cells[2],
                           bc=[3, 3, 2, 2, 1, 1], lat=0, level=level, group=group))

    for kb in range(nb[2]):
        for jb in range(nb[1]):
            for ib in range(nb[0]):
                lo = (x1a + ib * hb[0], jb * hb[1], kb * hb[2])
                polar = jb in (0, nb[1] - 1)
                half = (hb[0] / 2, hb[1] / 2, hb[2] / 2)
                if polar and ib in polar_split:
                    for jc in range(2):
                        for ic in range(2):
                            clo = (lo[0] + ic * half[0], lo[1] + jc * half[1])
                            if (jb == 0 and jc == 0) or (jb == nb[1] - 1 and jc == 1):
                                add((clo[0], clo[1], lo[2]), (half[0], half[1], hb[2]), axis_cells, 1,
                                    "polar child on the axis")
                            else:
                                for kc in range(2):
                                    add((clo[0], clo[1], lo[2] + kc * half[2]), half, far_cells, 1,
                                        "polar child off the axis")
                elif polar:
                    add(lo, hb, polar_cells, 0, "polar base")
                elif (ib, jb) in disk:
                    q = (hb[0] / 4, hb[1] / 4, hb[2] / 4)
                    for kc in range(2):
                        for jc in range(2):
                            for ic in range(2):
                                i1, j1, k1 = 2 * ib + ic, 2 * jb + jc, 2 * kb + kc
                                clo = (x1a + i1 * half[0], j1 * half[1], k1 * half[2])
                                if (i1, j1) in level2:
                                    for kf in range(2):
                                        for jf in range(2):
                                            for i_f in range(2):
                                                add((clo[0] + i_f * q[0], clo[1] + jf * q[1], clo[2] + kf * q[2]),
                                                    q, (n, n, n), 2, "level 2")
                                else:
                                    add(clo, half, (n, n, n), 1, "level 1")
                else:
                    add(lo, hb, (n, n, n), 0, "base")
    _mark_block_faces(blocks, periodic=(False, False, True))
    return blocks


def nesting_violations(blocks, period3=2.0 * math.pi):
    """Pairs of blocks that share a face or an edge (Sec. 3.2 names faces and edges; corners are not
    constrained) whose cell widths differ by more than a factor 2 in some direction:
    [(a, b, direction, ratio)]."""
    boxes = [_box(b) for b in blocks]
    h = [(b["dx1"], b["dx2"], b["dx3"]) for b in blocks]
    out = []
    for a in range(len(blocks)):
        la, ha = boxes[a]
        for c in range(a + 1, len(blocks)):
            lc, hc = boxes[c]
            overlap = 0
            touch = 0
            for d in range(3):
                tol = 1e-9 * max(ha[d] - la[d], hc[d] - lc[d])
                shifts = (-period3, 0.0, period3) if d == 2 else (0.0,)
                best = None
                for sft in shifts:
                    lo_, hi_ = max(la[d], lc[d] + sft), min(ha[d], hc[d] + sft)
                    if hi_ > lo_ + tol:
                        best = "overlap"
                        break
                    if abs(hi_ - lo_) <= tol:
                        best = "touch"
                if best is None:
                    break
                overlap += best == "overlap"
                touch += best == "touch"
            else:
                if touch >= 1 and overlap >= 1:          # a shared face (2 overlaps) or edge (1 overlap)
                    for d in range(3):
                        r = max(h[a][d], h[c][d]) / min(h[a][d], h[c][d])
                        if r > 2.0 + 1e-9:
                            out.append((a, c, d + 1, r))
    return out


def c3_tree(rin=1.2, rout=50.0, n=32, smr=0):
    """The 512-block torus tree of the batched AMR/LAT configuration (C3): a base of 8 x 4 x 4 blocks;
    the 16 disk blocks (r index 3-4, theta index 1-2) refined to level 1, the 16 level-1 blocks at
    global r index 8, theta index 3-4 refined to level 2 (the finest level: a 1024 x 512 x 512
    effective grid at n = 32); the 32 polar base blocks at r index 2-5 split 6-way; the polar base
    rows derefined in phi. Cell counts: base and levels 1-2 n^3, polar blocks n x n x n/2
    (13,107,200 cells at n = 32). Checked: no face or edge neighbours more than a factor 2 apart
    in any direction; LAT levels from assign_lat_levels (with smr internal SMR levels: the grouped
    polar rows' wider cells in phi)."""
    blocks = c3_blocks(n=n, rin=rin, rout=rout)
    bad = nesting_violations(blocks)
    if bad:
        raise ValueError("C3 tree violates the nesting rule: %s" % bad[:4])
    return assign_lat_levels(blocks, smr=smr)


def tree_summary(blocks):
    """Counts per group and shape, cells, LAT-level and refinement-level histograms."""
    groups = {}
    for b in blocks:
        key = "%s %dx%dx%d" % (b.get("group", "block"), b["n1"], b["n2"], b["n3"])
        groups[key] = groups.get(key, 0) + 1
    lat = {}
    lev = {}
    for b in blocks:
        lat[b["lat"]] = lat.get(b["lat"], 0) + 1
        lev[b.get("level", 0)] = lev.get(b.get("level", 0), 0) + 1
    return dict(blocks=len(blocks), cells=int(sum(b["n1"] * b["n2"] * b["n3"] for b in blocks)), groups=groups,
                lat_levels={str(k): v for k, v in sorted(lat.items())},
                refinement_levels={str(k): v for k, v in sorted(lev.items())})


def _softplus(x):
    return np.where(x > 30.0, x, np.log1p(np.exp(np.minimum(x, 30.0))))


def explosion_blocks(blocks, centre=(3.0, 0.0, 10.0), rs=2.0, rho=1e-4, p_in=3e-5, p_out=3e-8, width=0.1,
                     beta_max=None, gam=5.0 / 3.0, nquad=16):
    """An off-centre explosion in flat space on log-r spherical blocks (Sec. 6): density rho
    everywhere, pressure p_in inside the sphere of radius rs about the Cartesian point `centre` and
    p_out outside, joined by p_out + (p_in - p_out) / (1 + exp((d - rs) / (width rs))) (the smoothed
    edge; the ambient pressure is not given, p_out is this stand-in's choice), at rest. With
    beta_max, a field from the vector potential A_phi = c w rs ln(1 + exp((rs - d) / (w rs))) (the
    (rs - d) profile inside, 0 outside, with a smooth edge), its face fluxes from Gauss-Legendre
    integrals of A_phi along the phi-edges (divergence-free; a coarse edge integral is the sum of its
    fine ones to rounding), c set so that max p_gas / max p_mag = beta_max over the cells (flat
    space at rest: b^2 = r^2 (B^1)^2 + r^2 (B^2)^2, B^i = Bbar^i / (r^3 sin theta)). Returns padded
    (prim, bface) per block."""
    x0 = np.asarray(centre, dtype=float)
    gl_x, gl_w = np.polynomial.legendre.leggauss(nquad)

    def dist(r, th, ph):
        return np.sqrt((r * np.sin(th) * np.cos(ph) - x0[0]) ** 2 + (r * np.sin(th) * np.sin(ph) - x0[1]) ** 2
                       + (r * np.cos(th) - x0[2]) ** 2)

    out = []
    for b in blocks:
        n1, n2, n3 = b["n1"], b["n2"], b["n3"]
        shp = (n3 + 2 * NG, n2 + 2 * NG, n1 + 2 * NG)
        prim = np.zeros((8,) + shp)
        bf = np.zeros((3,) + shp)
        x1 = _centres(b["x1min"], b["dx1"], n1)
        x2 = _centres(b["x2min"], b["dx2"], n2)
        x3 = _centres(b["x3min"], b["dx3"], n3)
        P3, T2, R1 = np.meshgrid(x3, x2, np.exp(x1), indexing="ij")
        d = dist(R1, T2, P3)
        s = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
        prim[0][s] = rho
        prim[1][s] = (p_out + (p_in - p_out) / (1.0 + np.exp(np.minimum((d - rs) / (width * rs), 50.0)))) / (gam - 1.0)
        if beta_max is not None:
            # integrals of A_phi (unit c) along the phi-edges at the (x1, x2) corners
            xe1 = _edges(b["x1min"], b["dx1"], n1)
            xe2 = _edges(b["x2min"], b["dx2"], n2)
            I = np.zeros((n3, n2 + 1, n1 + 1))
            for k in range(n3):
                ph = b["x3min"] + (k + 0.5 + 0.5 * gl_x) * b["dx3"]
                E2, E1, PH = np.meshgrid(xe2, np.exp(xe1), ph, indexing="ij")
                dd = dist(E1, E2, PH)
                A = width * rs * _softplus((rs - dd) / (width * rs))
                I[k] = (A * (0.5 * b["dx3"] * gl_w)).sum(axis=2)
            bf[0][NG:NG + n3, NG:NG + n2, NG:NG + n1 + 1] = (I[:, 1:, :] - I[:, :-1, :]) / (b["dx2"] * b["dx3"])
            bf[1][NG:NG + n3, NG:NG + n2 + 1, NG:NG + n1] = -(I[:, :, 1:] - I[:, :, :-1]) / (b["dx1"] * b["dx3"])
        out.append((prim, bf))
    if beta_max is not None:
        pg, pb = 0.0, 0.0
        for b, (prim, bf) in zip(blocks, out):
            n1, n2, n3 = b["n1"], b["n2"], b["n3"]
            x1 = _centres(b["x1min"], b["dx1"], n1)
            x2 = _centres(b["x2min"], b["dx2"], n2)
            T2, R1 = np.meshgrid(x2, np.exp(x1), indexing="ij")
            gdet = R1 ** 3 * np.abs(np.sin(T2))
            b1 = 0.5 * (bf[0][NG:NG + n3, NG:NG + n2, NG:NG + n1] + bf[0][NG:NG + n3, NG:NG + n2, NG + 1:NG + n1 + 1])
            b2 = 0.5 * (bf[1][NG:NG + n3, NG:NG + n2, NG:NG + n1] + bf[1][NG:NG + n3, NG + 1:NG + n2 + 1, NG:NG + n1])
            bsq = R1 ** 2 * ((b1 / gdet) ** 2 + (b2 / gdet) ** 2)
            pb = max(pb, 0.5 * float(bsq.max()))
            pg = max(pg, float((gam - 1.0) * prim[1][NG:NG + n3, NG:NG + n2, NG:NG + n1].max()))
        c = math.sqrt(pg / (beta_max * pb)) if pb > 0 else 0.0
        for prim, bf in out:
            bf *= c
    return out


# --- tilted thin disk --------------------------------------------------------

def disk_geometry(n1=448, n2=192, n3=384, rin=1.2, rout=200.0):
    return BlockGeometry(n1, n2, n3, math.log(rin), math.log(rout), 0.0, math.pi, 0.0, 2.0 * math.pi)


def _trig_theta(th):
    """sin, cos of theta with the polar axis (0 or pi) mapped to exactly 0, +-1."""
    s, c = np.sin(th), np.cos(th)
    ax0 = np.abs(th) < 1e-12
    ax1 = np.abs(th - math.pi) < 1e-12
    s = np.where(ax0 | ax1, 0.0, s)
    c = np.where(ax0, 1.0, np.where(ax1, -1.0, c))
    return s, c


def tilted_disk_block(geo, a=0.9375, gam=13.0 / 9.0, hr=0.03, tilt_deg=65.0, beta=10.0, rd_in=6.0,
                      rd_out=100.0, pert=0.02, seed=4):
    """Padded primitive (8, n3p, n2p, n1p) and face-B (3, ...) arrays of a thin
    disk whose midplane is tilted by tilt_deg about the x axis.

    In the disk frame (normal n = (0, -sin tilt, cos tilt), height
    z' = r_vec . n, cylindrical radius R' = |r_vec - z' n|, scale height
    H = hr R'):
      rho = R'^-3/2 exp(-z'^2 / 2H^2) T(R'),  T = exp(-(rd_in/R')^6 - (R'/rd_out)^6),
      normalised to max rho = 1;
      p_g = rho c_s^2 / Gamma with c_s = hr v_K, v_K = R'^-1/2 (u_g = p_g/(Gamma-1)),
      with a seeded +/- pert perturbation of u_g;
      rotation at Omega = R'^-3/2 about n: coordinate velocity V = Omega n x r_vec
      (purely tangential, so dr/dt = 0), u^t from the metric normalisation and
      utilde^i = u^i + alpha^2 u^t g^{ti}; velocities only where the disk
      density exceeds 1e-6 of its maximum and r > 3.
    Field: toroidal about n, from the edge vector potential A = A_R' R'_hat with
    A_R' = sqrt(pi) H sqrt(2 p_mid(R')/beta) erf(z' / 2H), so that
    B_phi' = dA_R'/dz' = sqrt(2 p_g / beta) locally; face fluxes are the
    discrete curl of the covariant edge components (divergence-free to
    roundoff, zero on the polar axis), then normalised to
    max p_g / max p_b = beta over the block.
    Atmosphere and floors as in torus_block. Position geometry (r_vec, R', z')
    is flat-space spherical in (r, theta, phi).
    """
    n1, n2, n3 = geo.n1, geo.n2, geo.n3
    shp = geo.padded_shape
    prim = np.zeros((8,) + shp)
    bface = np.zeros((3,) + shp)
    tl = math.radians(tilt_deg)
    nvec = np.array([0.0, -math.sin(tl), math.cos(tl)])

    x1c = _centres(geo.x1min, geo.dx1, n1)
    x2c = _centres(geo.x2min, geo.dx2, n2)
    x3c = _centres(geo.x3min, geo.dx3, n3)
    x1e = _edges(geo.x1min, geo.dx1, n1)
    x2e = _edges(geo.x2min, geo.dx2, n2)
    x3e = _edges(geo.x3min, geo.dx3, n3)[:n3]  # phi edge n3 is edge 0 (periodic)

    def frame(r, th, ph):
        s, c = _trig_theta(th)
        cp, sp = np.cos(ph), np.sin(ph)
        rhat = np.stack(np.broadcast_arrays(s * cp, s * sp, c))
        thhat = np.stack(np.broadcast_arrays(c * cp, c * sp, -s))
        phhat = np.stack(np.broadcast_arrays(-sp, cp, 0.0 * s))
        rv = r * rhat
        zp = nvec[0] * rv[0] + nvec[1] * rv[1] + nvec[2] * rv[2]
        rperp = rv - zp * nvec[:, None, None]
        Rp = np.sqrt(np.maximum(r * r - zp * zp, 0.0))
        return s, rhat, thhat, phhat, rv, zp, rperp, Rp

    def taper(Rp):
        with np.errstate(divide="ignore", over="ignore"):
            return np.exp(-(rd_in / np.maximum(Rp, 1e-3)) ** 6 - (Rp / rd_out) ** 6)

    def rho_disk(Rp, zp):
        Rs = np.maximum(Rp, 1e-3)
        H = hr * Rs
        return Rs ** -1.5 * np.exp(-zp * zp / (2.0 * H * H)) * taper(Rp)

    # normalisation: the maximum sits on the midplane, max over R' of R'^-3/2 T(R')
    Rg = np.exp(np.linspace(0.0, math.log(2.0 * rd_out), 20001))
    rho0 = float((Rg ** -1.5 * taper(Rg)).max())

    R2, TH2 = np.meshgrid(np.exp(x1c), x2c, indexing="xy")  # (n2, n1) centres
    gcov, gtt_con, gt1_con, gdet = _ks_internal(a, R2, TH2)
    alpha = 1.0 / np.sqrt(-gtt_con)
    rho_flr = 1.0e-7 / R2 ** 2
    u_flr = 1.0e-9 * R2 ** (-10.0 / 3.0)
    pgmax = 0.0
    sl = (slice(NG, NG + n2), slice(NG, NG + n1))
    for k in range(n3):
        s, rhat, thhat, phhat, rv, zp, rperp, Rp = frame(R2, TH2, x3c[k])
        rho_d = rho_disk(Rp, zp) / rho0
        cs2 = hr * hr / np.maximum(Rp, 1e-3)
        u_d = rho_d * cs2 / gam / (gam - 1.0)
        ids = (np.arange(n1)[None, :] + n1 * (np.arange(n2)[:, None] + n2 * k)).astype(np.uint64)
        xi = uniform01(seed, ids)
        disk = (rho_d > 1e-6) & (R2 > 3.0)
        u_d = np.where(disk, u_d * (1.0 + pert * (2.0 * xi - 1.0)), u_d)
        rho = np.maximum(rho_d, rho_flr)
        u = np.maximum(u_d, u_flr)
        # tilted Keplerian rotation, coordinate velocity dx^i/dt
        Om = np.maximum(Rp, 1e-3) ** -1.5
        V = Om * np.cross(nvec[:, None, None], rv, axis=0)
        V2 = (V * thhat).sum(axis=0) / R2
        V3 = np.where(s > 0.0, (V * phhat).sum(axis=0) / (R2 * np.where(s > 0.0, s, 1.0)), 0.0)
        norm = -(gcov[(0, 0)] + 2.0 * gcov[(0, 3)] * V3 + gcov[(2, 2)] * V2 * V2 + gcov[(3, 3)] * V3 * V3)
        ok = disk & (norm > 0.0)
        ut = np.where(ok, 1.0 / np.sqrt(np.where(ok, norm, 1.0)), 0.0)
        prim[0, NG + k][sl] = rho
        prim[1, NG + k][sl] = u
        prim[2, NG + k][sl] = np.where(ok, alpha * alpha * ut * gt1_con, 0.0)
        prim[3, NG + k][sl] = ut * V2
        prim[4, NG + k][sl] = ut * V3
        pgmax = max(pgmax, float(((gam - 1.0) * u).max()))

    # edge vector potential, covariant components in (x1, x2, x3)
    def a_cov(r, th, ph, comp):
        s, rhat, thhat, phhat, rv, zp, rperp, Rp = frame(r, th, ph)
        Rs = np.maximum(Rp, 1e-3)
        H = hr * Rs
        pmid = Rs ** -1.5 * taper(Rp) / rho0 * (hr * hr / Rs) / gam
        amp = math.sqrt(math.pi) * H * np.sqrt(2.0 * pmid / beta) * _erf(zp / (2.0 * H))
        Rhat = rperp / Rs
        e = (rhat * r, thhat * r, phhat * (r * s))[comp]
        return amp * (Rhat * e).sum(axis=0)

    A1 = np.empty((n3, n2 + 1, n1))
    A2 = np.empty((n3, n2, n1 + 1))
    A3 = np.empty((n3, n2 + 1, n1 + 1))
    Rc1, Te1 = np.meshgrid(np.exp(x1c), x2e, indexing="xy")
    Re2, Tc2 = np.meshgrid(np.exp(x1e), x2c, indexing="xy")
    Re3, Te3 = np.meshgrid(np.exp(x1e), x2e, indexing="xy")
    for k in range(n3):
        A1[k] = a_cov(Rc1, Te1, x3e[k], 0)
        A2[k] = a_cov(Re2, Tc2, x3e[k], 1)
        A3[k] = a_cov(Re3, Te3, x3c[k], 2)
    A1p = np.concatenate([A1, A1[:1]], axis=0)  # edge k = n3 is edge 0
    A2p = np.concatenate([A2, A2[:1]], axis=0)
    # Bbar^1 = d2 A3 - d3 A2 at x1 faces (n3, n2, n1+1)
    b1 = (A3[:, 1:, :] - A3[:, :-1, :]) / geo.dx2 - (A2p[1:] - A2p[:-1]) / geo.dx3
    # Bbar^2 = d3 A1 - d1 A3 at x2 faces (n3, n2+1, n1)
    b2 = (A1p[1:] - A1p[:-1]) / geo.dx3 - (A3[:, :, 1:] - A3[:, :, :-1]) / geo.dx1
    # Bbar^3 = d1 A2 - d2 A1 at x3 faces (n3, n2, n1)
    b3 = (A2[:, :, 1:] - A2[:, :, :-1]) / geo.dx1 - (A1[:, 1:, :] - A1[:, :-1, :]) / geo.dx2
    if geo.x2min == 0.0:
        b2[:, 0, :] = 0.0
    if abs(geo.x2min + n2 * geo.dx2 - math.pi) < 1e-12:
        b2[:, -1, :] = 0.0

    # normalise to max p_g / max p_b = beta with centre B = <Bbar>/sqrt(-g)
    pbmax = 0.0
    for k in range(n3):
        kp = (k + 1) % n3
        Bc1 = 0.5 * (b1[k, :, :-1] + b1[k, :, 1:]) / gdet
        Bc2 = 0.5 * (b2[k, :-1, :] + b2[k, 1:, :]) / gdet
        Bc3 = 0.5 * (b3[k] + b3[kp]) / gdet
        pu = (prim[2, NG + k][sl], prim[3, NG + k][sl], prim[4, NG + k][sl])
        pbmax = max(pbmax, float(0.5 * _bsq(a, R2, TH2, pu, (Bc1, Bc2, Bc3)).max()))
    fac = math.sqrt(pgmax / (beta * pbmax)) if (pbmax > 0.0 and beta > 0.0) else 0.0
    bface[0, NG:NG + n3, NG:NG + n2, NG:NG + n1 + 1] = fac * b1
    bface[1, NG:NG + n3, NG:NG + n2 + 1, NG:NG + n1] = fac * b2
    bface[2, NG:NG + n3, NG:NG + n2, NG:NG + n1] = fac * b3
    return prim, bface


def _erf(x):
    """Vectorised error function (scipy when present, else math.erf per element)."""
    try:
        from scipy.special import erf as serf
        return serf(x)
    except ImportError:  # pragma: no cover
        return np.vectorize(math.erf)(x)


# --- spherical accretion ------------------------------------------------------

def _bondi_theta(c2, gam):
    """Theta = p/rho of a polytrope with sound speed squared c2 (c2 = gam Theta / h, h = 1 + gam Theta/(gam - 1))."""
    return c2 / (gam * (1.0 - c2 / (gam - 1.0)))


def bondi_profile(r, rc=8.0, gam=4.0 / 3.0, rho_c=1.0):
    """Relativistic spherical accretion onto a Schwarzschild hole (Michel 1972), M = 1.

    Sonic point rc: u_c^2 = 1/(2 rc), c_s^2 = u_c^2 / (1 - 3 u_c^2). Along the
    flow rho u r^2 and h^2 (1 - 2/r + u^2) are constant (u = -u^r > 0, the
    radial 4-velocity, the same in Schwarzschild and Kerr-Schild time), and
    p = K rho^gam. Returns rho, u (inflow speed u = -u^r) and Theta = p/rho
    at radii r (the subsonic root outside rc, the supersonic one inside).
    """
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    uc2 = 1.0 / (2.0 * rc)
    cs2 = uc2 / (1.0 - 3.0 * uc2)
    th_c = _bondi_theta(cs2, gam)
    K = th_c / rho_c ** (gam - 1.0)
    uc = math.sqrt(uc2)
    mdot = rho_c * uc * rc * rc
    hc = 1.0 + gam * th_c / (gam - 1.0)
    bern = hc * hc * (1.0 - 2.0 / rc + uc2)

    def f(lnrho, rr):
        rho = math.exp(lnrho)
        th = K * rho ** (gam - 1.0)
        h = 1.0 + gam * th / (gam - 1.0)
        u = mdot / (rho * rr * rr)
        return h * h * (1.0 - 2.0 / rr + u * u) - bern

    out_rho = np.empty_like(r)
    for n, rr in enumerate(r):
        # f(ln rho) is convex in ln rho with its minimum at the sonic condition; bracket both roots
        lo, hi = math.log(rho_c) - 40.0, math.log(rho_c) + 40.0
        a, b = lo, hi
        for _ in range(200):  # golden-section search for the minimum
            m1 = a + 0.381966 * (b - a)
            m2 = b - 0.381966 * (b - a)
            if f(m1, rr) < f(m2, rr):
                b = m2
            else:
                a = m1
        xm = 0.5 * (a + b)
        if abs(rr - rc) < 1e-12:
            out_rho[n] = math.exp(xm)
            continue
        a, b = (xm, hi) if rr > rc else (lo, xm)  # subsonic (denser) outside, supersonic inside
        fa = f(a, rr)
        for _ in range(200):  # bisection
            mid = 0.5 * (a + b)
            fm = f(mid, rr)
            if (fm > 0) == (fa > 0):
                a, fa = mid, fm
            else:
                b = mid
        out_rho[n] = math.exp(0.5 * (a + b))
    th = K * out_rho ** (gam - 1.0)
    u = mdot / (out_rho * r * r)
    return out_rho, u, th


def bondi_block(geo, rc=8.0, gam=4.0 / 3.0):
    """Padded primitive and (zero) face-B arrays of the Michel solution on a
    Kerr-Schild a = 0 block (x1 = log r): rho, u_g = p/(gam - 1) and
    utilde^1 = u^1 + alpha^2 u^t g^{t1} with u^1 = u^r / r, u^t from the
    normalisation; utilde^2 = utilde^3 = 0."""
    n1, n2, n3 = geo.n1, geo.n2, geo.n3
    prim = np.zeros((8,) + geo.padded_shape)
    bface = np.zeros((3,) + geo.padded_shape)
    # every cell of the padded block (ghosts too: the x1 ghosts then start at the solution)
    x1 = geo.x1min + (np.arange(-NG, n1 + NG) + 0.5) * geo.dx1
    r = np.exp(x1)
    rho, u, th = bondi_profile(r, rc=rc, gam=gam)
    # Kerr-Schild a = 0 in (t, log r): g_tt = -(1 - 2/r), g_t1 = 2, g_11 = (1 + 2/r) r^2; g^tt = -(1 + 2/r), g^t1 = 2/r^2
    u1 = -u / r
    A, Bq, Cq = -(1.0 - 2.0 / r), 2.0 * 2.0 * u1, (1.0 + 2.0 / r) * r * r * u1 * u1 + 1.0
    ut = (-Bq - np.sqrt(Bq * Bq - 4.0 * A * Cq)) / (2.0 * A)
    alpha2 = 1.0 / (1.0 + 2.0 / r)
    ut1 = u1 + alpha2 * ut * (2.0 / (r * r))
    prim[0] = rho[None, None, :]
    prim[1] = (rho * th / (gam - 1.0))[None, None, :]
    prim[2] = ut1[None, None, :]
    return prim, bface


# --- field-loop advection (flat space) ------------------------------------------

def field_loop_block(n1, n2, n3=4, L=1.0, R=0.3, A0=1e-3, rho=1.0, p=0.1, v=(0.4, 0.2), gam=5.0 / 3.0):
    """A weak cylindrical field loop (A_3 = A0 (R - r) inside r < R, r from the box centre) in a
    uniform flow with 3-velocity v in a periodic L x L box (x1, x2; n3 cells of size 1 along x3).
    Face B is the discrete curl of A_3 at the x3-edges (divergence-free to round-off); returns
    the padded primitive and face arrays and the cell sizes."""
    dx1, dx2 = L / n1, L / n2
    shp = (n3 + 2 * NG, n2 + 2 * NG, n1 + 2 * NG)
    prim = np.zeros((8,) + shp)
    bface = np.zeros((3,) + shp)
    W = 1.0 / math.sqrt(1.0 - v[0] * v[0] - v[1] * v[1])
    prim[0][...] = rho
    prim[1][...] = p / (gam - 1.0)
    prim[2][...] = W * v[0]
    prim[3][...] = W * v[1]
    xe = np.arange(n1 + 1) * dx1 - 0.5 * L
    ye = np.arange(n2 + 1) * dx2 - 0.5 * L
    X, Y = np.meshgrid(xe, ye, indexing="xy")  # edges (i-1/2, j-1/2): (n2+1, n1+1)
    r = np.sqrt(X * X + Y * Y)
    A = np.where(r < R, A0 * (R - r), 0.0)
    b1 = (A[1:, :] - A[:-1, :]) / dx2        # Bbar^1 = dA3/dx2 on x1 faces i = 0..n1: (n2, n1+1)
    b2 = -(A[:, 1:] - A[:, :-1]) / dx1       # Bbar^2 = -dA3/dx1 on x2 faces j = 0..n2: (n2+1, n1)
    for k in range(n3):
        bface[0, NG + k, NG:NG + n2, NG:NG + n1 + 1] = b1
        bface[1, NG + k, NG:NG + n2 + 1, NG:NG + n1] = b2
    return prim, bface, dx1, dx2


def riemann_block(n1, left, right, n2=4, n3=4, x0=0.5, gam=5.0 / 3.0):
    """A one-dimensional Riemann problem along x1 of a unit flat-space box: states (rho, p, v) left
    and right of x = x0 (v the x1 3-velocity), uniform across x2 and x3 (n2 x n3 cells). Returns
    the padded primitive array and zero face B."""
    shp = (n3 + 2 * NG, n2 + 2 * NG, n1 + 2 * NG)
    prim = np.zeros((8,) + shp)
    x = (np.arange(-NG, n1 + NG) + 0.5) / n1
    on_left = x < x0
    for q, (a, b) in enumerate([(left[0], right[0]), (left[1] / (gam - 1.0), right[1] / (gam - 1.0)),
                                (left[2] / math.sqrt(1.0 - left[2] ** 2), right[2] / math.sqrt(1.0 - right[2] ** 2))]):
        prim[q][...] = np.where(on_left, a, b)[None, None, :]
    return prim, np.zeros((3,) + shp)


def _edge_integral(c, k, h, phase):
    """Integral over s in [0, h] of c cos(phase + k s)."""
    if abs(k * h) < 1e-12:
        return c * h * np.cos(phase)
    return c * (np.sin(phase + k * h) - np.sin(phase)) / k


def linear_wave_states(blocks, rho0, p0, B0, kvec, R, r, amp, gam=5.0 / 3.0):
    """A plane linear wave on flat-space blocks: background rho0, p0 at rest with uniform field B0
    (3-vector), perturbation amp * r * sin(k.x) where r is a given eigenvector in the wave's frame,
    r = (drho, dp, dv_par, dv_perp1, dv_perp2, dB_perp1, dB_perp2), and R the rotation whose
    columns are the wave frame's axes (R[:, 0] = k / |k|) in grid coordinates. Face B is B0 plus the
    face average of the curl of the vector potential (k x b) / |k|^2 cos(k.x), b = amp R (0, dB1, dB2),
    taken from exact edge integrals (divergence-free, and a coarse face's flux is the sum of its fine
    faces'). Returns [(prim, bface)] per block (padded; ghosts left for the library)."""
    kvec = np.asarray(kvec, dtype=float)
    k2 = kvec @ kvec
    b = amp * (R @ np.array([0.0, r[5], r[6]]))
    cvec = np.cross(kvec, b) / k2
    dv = amp * (R @ np.array([r[2], r[3], r[4]]))
    out = []
    for blk in blocks:
        n1, n2, n3 = blk["n1"], blk["n2"], blk["n3"]
        h = (blk["dx1"], blk["dx2"], blk["dx3"])
        lo = (blk["x1min"], blk["x2min"], blk["x3min"])
        shp = (n3 + 2 * NG, n2 + 2 * NG, n1 + 2 * NG)
        prim = np.zeros((8,) + shp)
        bf = np.zeros((3,) + shp)
        x = _centres(lo[0], h[0], n1)
        y = _centres(lo[1], h[1], n2)
        z = _centres(lo[2], h[2], n3)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        sn = np.sin(kvec[0] * X + kvec[1] * Y + kvec[2] * Z)
        s = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
        prim[0][s] = rho0 + amp * r[0] * sn
        prim[1][s] = (p0 + amp * r[1] * sn) / (gam - 1.0)
        v = [dv[d] * sn for d in range(3)]
        lor = 1.0 / np.sqrt(1.0 - (v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
        for d in range(3):
            prim[2 + d][s] = lor * v[d]
        xe = _edges(lo[0], h[0], n1)
        ye = _edges(lo[1], h[1], n2)
        ze = _edges(lo[2], h[2], n3)
        # x1 faces: circulation of A around (y0..y0+hy) x (z0..z0+hz) at x = xe
        Zc, Yc, Xe = np.meshgrid(ze[:-1], ye[:-1], xe, indexing="ij")
        ph = kvec[0] * Xe + kvec[1] * Yc + kvec[2] * Zc
        Iy0 = _edge_integral(cvec[1], kvec[1], h[1], ph)
        Iy1 = _edge_integral(cvec[1], kvec[1], h[1], ph + kvec[2] * h[2])
        Iz0 = _edge_integral(cvec[2], kvec[2], h[2], ph)
        Iz1 = _edge_integral(cvec[2], kvec[2], h[2], ph + kvec[1] * h[1])
        bf[0][NG:NG + n3, NG:NG + n2, NG:NG + n1 + 1] = B0[0] + ((Iy0 - Iy1) + (Iz1 - Iz0)) / (h[1] * h[2])
        # x2 faces: (z, x) circulation at y = ye: B2 = dA1/dz - dA3/dx
        Zc, Ye, Xc = np.meshgrid(ze[:-1], ye, xe[:-1], indexing="ij")
        ph = kvec[0] * Xc + kvec[1] * Ye + kvec[2] * Zc
        Iz0 = _edge_integral(cvec[2], kvec[2], h[2], ph)
        Iz1 = _edge_integral(cvec[2], kvec[2], h[2], ph + kvec[0] * h[0])
        Ix0 = _edge_integral(cvec[0], kvec[0], h[0], ph)
        Ix1 = _edge_integral(cvec[0], kvec[0], h[0], ph + kvec[2] * h[2])
        bf[1][NG:NG + n3, NG:NG + n2 + 1, NG:NG + n1] = B0[1] + ((Iz0 - Iz1) + (Ix1 - Ix0)) / (h[2] * h[0])
        # x3 faces: (x, y) circulation at z = ze: B3 = dA2/dx - dA1/dy
        Ze, Yc, Xc = np.meshgrid(ze, ye[:-1], xe[:-1], indexing="ij")
        ph = kvec[0] * Xc + kvec[1] * Yc + kvec[2] * Ze
        Ix0 = _edge_integral(cvec[0], kvec[0], h[0], ph)
        Ix1 = _edge_integral(cvec[0], kvec[0], h[0], ph + kvec[1] * h[1])
        Iy0 = _edge_integral(cvec[1], kvec[1], h[1], ph)
        Iy1 = _edge_integral(cvec[1], kvec[1], h[1], ph + kvec[0] * h[0])
        bf[2][NG:NG + n3 + 1, NG:NG + n2, NG:NG + n1] = B0[2] + ((Ix0 - Ix1) + (Iy1 - Iy0)) / (h[0] * h[1])
        out.append((prim, bf))
    return out
