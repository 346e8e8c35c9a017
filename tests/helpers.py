"""Shared set-up of the parity tests: the same seeded state fed to the CUDA
library (through its C ABI) and to the CPU oracle."""
import numpy as np

import oracle as O
from paper_1912_10192_gb300 import workloads as W

NG = 3
TORUS_BC = (O.BC_OUTFLOW_NOINFLOW, O.BC_OUTFLOW_NOINFLOW, O.BC_POLAR, O.BC_POLAR, O.BC_PERIODIC, O.BC_PERIODIC)


def torus_case(n1, n2, n3, seed, a=0.9375, gam=13.0 / 9.0, cour=0.8, recon=O.RECON_PPM, riemann=O.FLUX_HLL,
               beta=100.0):
    geo = W.torus_geometry(n1, n2, n3)
    prim, bf = W.torus_block(geo, a=a, gam=gam, seed=seed, beta=beta)
    d = O.make_desc(n1, n2, n3, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3, metric=O.METRIC_KS,
                    a=a, gam=gam, cour=cour, recon=recon, riemann=riemann, bc=TORUS_BC)
    return geo, d, prim, bf


def gpu_grid(d):
    from paper_1912_10192_gb300 import hamr
    b = hamr.block(d.n1, d.n2, d.n3, d.x1min, d.x2min, d.x3min, d.dx1, d.dx2, d.dx3, tuple(d.bc))
    return hamr.Grid([b], metric=d.metric, a=d.a, gam=d.gam, cour=d.cour, recon=d.recon, riemann=d.riemann,
                     floors=d.floors, emf=d.emf, flatten=d.flatten,
                     inversion=d.inversion, floor_frame=d.floor_frame, smr=d.smr)


def interior(a, d):
    return a[..., NG:NG + d.n3, NG:NG + d.n2, NG:NG + d.n1]


def face_interior(bf, d):
    """The faces both codes evolve: Bbar^1 on i = 0..n1, Bbar^2 on j = 0..n2, Bbar^3 on k = 0..n3."""
    s = NG
    return [bf[0][s:s + d.n3, s:s + d.n2, s:s + d.n1 + 1],
            bf[1][s:s + d.n3, s:s + d.n2 + 1, s:s + d.n1],
            bf[2][s:s + d.n3 + 1, s:s + d.n2, s:s + d.n1]]


def rel_l1(x, ref):
    den = np.abs(ref).sum()
    num = np.abs(x - ref).sum()
    return num / den if den > 0 else num


def inversion_bar(d, U, B, x1, x2, p_ref, p_exact, safety=32.0, p_other=None):
    """Per state and primitive: how far a correct energy inversion of the conserved state U may lie
    from the reference result p_ref, given the conditioning of the inversion.

    With J = dU/dP (the FP64 prim -> cons map over the five hydro primitives at fixed B, by central
    differences of the oracle's map at p_ref), two inversions whose residuals U(p) - U are both at the
    rounding level s of evaluating that map differ by at most sum_m |J^-1|_im 2 s_m to first order.
    s_m is estimated from two points where the map's value is known to be U up to its own rounding:
    the reference result and the primitives U was formed from (p_exact), floored at the unit
    round-off of U_m. A candidate with a larger residual (a wrong root, a dropped term) is not
    covered by the bar. For an iteration that stops at a tolerance rather than at round-off (the
    Aitken pressure iteration), pass the candidate as p_other: its own residual then enters s, and
    the caller bounds that residual (its backward error) separately. Returns (n, 5) absolute bars."""
    import oracle as O
    n = U.shape[0]
    J = np.zeros((n, 5, 5))
    vscale = np.maximum(np.abs(p_ref[:, 2:5]).max(axis=1), 1e-300)
    for v in range(5):
        h = 1e-6 * (np.maximum(np.abs(p_ref[:, v]), 1e-300) if v < 2 else vscale)
        pp, pm = p_ref.copy(), p_ref.copy()
        pp[:, v] += h
        pm[:, v] -= h
        J[:, :, v] = (O.p2u_many(d, pp, x1, x2)[:, :5] - O.p2u_many(d, pm, x1, x2)[:, :5]) / (2 * h)[:, None]
    Ji = np.abs(np.linalg.inv(J))
    eps = np.finfo(np.float64).eps
    pr, pe = p_ref.copy(), p_exact.copy()
    pr[:, 5:8] = B
    pe[:, 5:8] = B
    s = np.maximum(np.abs(O.p2u_many(d, pr, x1, x2)[:, :5] - U[:, :5]),
                   np.abs(O.p2u_many(d, pe, x1, x2)[:, :5] - U[:, :5]))
    if p_other is not None:
        po = p_other.copy()
        po[:, 5:8] = B
        s = np.maximum(s, np.abs(O.p2u_many(d, po, x1, x2)[:, :5] - U[:, :5]))
    s = np.maximum(s, eps * np.abs(U[:, :5]))
    return safety * np.einsum("nim,nm->ni", Ji, 2.0 * s)


U32 = 2.0 ** -24


def mixed_rounding_per_step(d, prim, bf):
    """A-priori size of one step's FP32 rounding in the mixed form, per field, relative L1.

    Each face flux computed from FP32 edge values carries a relative error of order the FP32 unit
    round-off u: a cell's conserved state then moves by up to u sum over its 6 faces of
    dt/dx |F_m| per component m (the oracle's own first-stage fluxes of the state, at the CFL dt),
    which the inversion maps to the primitives through |J^-1| (J = dU/dP of the FP64 prim -> cons
    map); the face field moves by u dt/dx times its EMFs (the B rows of the fluxes). Returns
    {rho, u, utilde, Bface}: sum over cells of the moved amount / sum |field|."""
    import oracle as O
    g = O.Grid(d)
    g.set(prim, bf)
    dt = g.dt()
    P, B = g.get()
    F = g.fluxes()
    n1, n2, n3 = d.n1, d.n2, d.n3
    s = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
    dx = (d.dx1, d.dx2, d.dx3)
    dU = np.zeros((5, n3, n2, n1))
    dB = np.zeros((n3, n2, n1))
    for dd in range(3):
        hi = [slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1)]
        hi[2 - dd] = slice(NG + 1, NG + 1 + (n1, n2, n3)[dd])
        for m in range(5):
            dU[m] += dt / dx[dd] * (np.abs(F[dd, m][s]) + np.abs(F[dd, m][tuple(hi)]))
        for m in (6, 7):
            dB += dt / dx[dd] * 2.0 * np.abs(F[dd, m][s])
    k, j, i = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    pr = np.stack([P[v][s].ravel() for v in range(8)], axis=1)
    x1 = d.x1min + (i.ravel() + 0.5) * d.dx1
    x2 = d.x2min + (j.ravel() + 0.5) * d.dx2
    J = np.zeros((len(x1), 5, 5))
    vs = np.maximum(np.abs(pr[:, 2:5]).max(axis=1), 1e-6)
    for v in range(5):
        h = 1e-6 * (np.maximum(np.abs(pr[:, v]), 1e-300) if v < 2 else vs)
        pp, pm = pr.copy(), pr.copy()
        pp[:, v] += h
        pm[:, v] -= h
        J[:, :, v] = (O.p2u_many(d, pp, x1, x2)[:, :5] - O.p2u_many(d, pm, x1, x2)[:, :5]) / (2 * h)[:, None]
    dP = np.einsum("nfm,nm->nf", np.abs(np.linalg.inv(J)), U32 * dU.reshape(5, -1).T)
    return {"rho": dP[:, 0].sum() / np.abs(pr[:, 0]).sum(), "u": dP[:, 1].sum() / np.abs(pr[:, 1]).sum(),
            "utilde": dP[:, 2:5].sum() / np.abs(pr[:, 2:5]).sum(),
            "Bface": U32 * dB.sum() / sum(np.abs(B[m][s]).sum() for m in range(3))}


def polar_field(bf, x1min, x2min, x3min, dx1, dx2, dx3, n, B0=1e-3, m3=0.3):
    """adds a divergence-free field threading the poles to the face fluxes bf (padded, in place): the
    vector potential A_3 = (B0 / 2) r^2 sin^2(theta) (1 + m3 cos phi) (r = exp(x1), theta = x2,
    phi = x3) at the cells' x3-edges (a vertical field, modulated in phi), whose discrete curl gives
    the x1- and x2-face fluxes of each phi cell"""
    n1, n2, n3 = n
    r = np.exp(x1min + np.arange(n1 + 1) * dx1)
    th = x2min + np.arange(n2 + 1) * dx2
    ph = x3min + (np.arange(n3) + 0.5) * dx3
    A = 0.5 * B0 * (r[None, None, :] * np.sin(th)[None, :, None]) ** 2 * (1.0 + m3 * np.cos(ph))[:, None, None]
    bf[0][NG:NG + n3, NG:NG + n2, NG:NG + n1 + 1] += (A[:, 1:, :] - A[:, :-1, :]) / dx2
    bf[1][NG:NG + n3, NG:NG + n2 + 1, NG:NG + n1] += -(A[:, :, 1:] - A[:, :, :-1]) / dx1


def polar_field_desc(bf, d, B0=1e-3, m3=0.3):
    """polar_field on the single block of descriptor d"""
    polar_field(bf, d.x1min, d.x2min, d.x3min, d.dx1, d.dx2, d.dx3, (d.n1, d.n2, d.n3), B0=B0, m3=m3)


def refined_polar_tree(n=8, nb=(4, 2, 2), centre=(1.0, 0.0, 18.0), B0=1e-8, gam=5.0 / 3.0):
    """flat log-r spherical blocks over r in [2, 40], the radial block column at index 2 refined
    (octants, 6-way next to the axis), LAT levels; an explosion over the axis across the face where
    the refined blocks meet a coarser block on a slower LAT level (refluxed cells in grouped rows),
    into a cold ambient (p = 1e-14, so the discrete imbalance of a gas at rest in spherical
    coordinates moves no measurable mass through the radial boundaries), plus a weak axisymmetric
    vertical field through the poles. Returns (blocks, states)."""
    blocks = W.polar_smr_tree(2.0, 40.0, nb, n, range(2, 3))
    states = W.explosion_blocks(blocks, centre=centre, gam=gam, p_out=1e-14)
    for b, (p, bf) in zip(blocks, states):
        polar_field(bf, b["x1min"], b["x2min"], b["x3min"], b["dx1"], b["dx2"], b["dx3"],
                    (b["n1"], b["n2"], b["n3"]), B0=B0, m3=0.0)
    return blocks, states


def ora_tree(phys, blocks, states):
    """the oracle's multi-block grid of block dicts with their padded states"""
    a = O.AmrGrid(phys, [O.make_block(b["n1"], b["n2"], b["n3"], b["x1min"], b["x2min"], b["x3min"], b["dx1"],
                                      b["dx2"], b["dx3"], b["bc"], b["lat"]) for b in blocks])
    for i, (p, bf) in enumerate(states):
        a.set(i, p, bf)
    return a


def tree_errors(g, a, blocks):
    """relative L1 differences (rho, u, utilde, face fluxes) between the GPU grid g and the oracle's a
    over the interiors of all blocks"""
    num = {k: 0.0 for k in ("rho", "u", "utilde", "Bface")}
    den = dict(num)
    for i, b in enumerate(blocks):
        pg, bg = g.get_state(block=i)
        po, bo = a.get(i)
        n1, n2, n3 = b["n1"], b["n2"], b["n3"]
        s = (slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1))
        for k, vs in (("rho", (0,)), ("u", (1,)), ("utilde", (2, 3, 4))):
            for v in vs:
                num[k] += np.abs(pg[v][s] - po[v][s]).sum()
                den[k] += np.abs(po[v][s]).sum()
        fs = [(slice(NG, NG + n3), slice(NG, NG + n2), slice(NG, NG + n1 + 1)),
              (slice(NG, NG + n3), slice(NG, NG + n2 + 1), slice(NG, NG + n1)),
              (slice(NG, NG + n3 + 1), slice(NG, NG + n2), slice(NG, NG + n1))]
        for m in range(3):
            num["Bface"] += np.abs(bg[m][fs[m]] - bo[m][fs[m]]).sum()
            den["Bface"] += np.abs(bo[m][fs[m]]).sum()
    return {k: num[k] / max(den[k], 1e-300) for k in num}
