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
