"""Pins of the face value of the entropy tracer. Sec. 2.1 evolves the conserved
entropy kappa rho u^mu beside the fluid but leaves kappa's value at a face
open; the oracle forms every cell's kappa = p / rho^gam and reconstructs it to
the faces like a primitive. Two consequences that fix this reading:

- in an isentropic state (one kappa everywhere) the entropy flux through every
  face is exactly kappa times the mass flux, whatever the reconstruction does
  to rho and u_g (p / rho^gam of the reconstructed rho and u_g would differ
  from kappa by the reconstruction's truncation error);
- in a flow faster than every wave HLL takes the upwind state alone, so the
  entropy flux over the mass flux is the upwind cell's reconstructed kappa
  (its right edge value for a flow along +x1), not the downwind cell's.
"""
import numpy as np

import oracle as O
from helpers import NG, torus_case
from paper_1912_10192_gb300 import workloads as W


def test_isentropic_state_carries_kappa_exactly():
    geo, d, prim, bf = torus_case(16, 16, 8, seed=7)
    kap0 = 0.02
    prim[1] = kap0 * prim[0] ** d.gam / (d.gam - 1.0)
    g = O.Grid(d)
    g.set(prim, bf)
    F = g.fluxes()
    mass, ent = F[:, 0], F[:, 5]
    assert np.abs(mass).max() > 0.0
    # per face: rounding of the few products that form each flux
    err = np.abs(ent - kap0 * mass)
    assert err.max() <= 1e-13 * kap0 * np.abs(mass).max()
    big = np.abs(mass) > 1e-6 * np.abs(mass).max()
    assert (err[big] <= 1e-12 * kap0 * np.abs(mass[big])).all()


def test_isentropic_pin_would_see_face_kappa_of_edge_primitives():
    """The first pin discriminates: on the same state, p / rho^gam of PPM edge values of rho and
    u_g differs from kappa far above the pin's tolerance."""
    geo, d, prim, bf = torus_case(16, 16, 8, seed=7)
    kap0 = 0.02
    prim[1] = kap0 * prim[0] ** d.gam / (d.gam - 1.0)
    g = O.Grid(d)
    g.set(prim, bf)
    g.bc()
    p, _ = g.get()
    worst = 0.0
    for k in range(NG, NG + d.n3):
        rl, rr = O.recon_line(O.RECON_PPM, p[0][k, NG + d.n2 // 2, :])
        ul, ur = O.recon_line(O.RECON_PPM, p[1][k, NG + d.n2 // 2, :])
        c = slice(NG - 1, NG + d.n1 + 1)
        kf = (d.gam - 1.0) * ur[c] / rr[c] ** d.gam
        worst = max(worst, np.abs(kf / kap0 - 1.0).max())
    assert worst > 1e-6


def test_supersonic_flow_takes_the_upwind_cells_kappa():
    n1, gam = 32, 5.0 / 3.0
    prim, bf = W.riemann_block(n1, (1.0, 1e-4, 0.9), (1.0, 1e-4, 0.9), gam=gam)
    x = (np.arange(-NG, n1 + NG) + 0.5) / n1
    # uniform pressure and velocity (v = 0.9, far above the sound speed ~0.02); rho, hence kappa,
    # varies smoothly and jumps at x = 0.6
    prim[0][...] = (1.0 + 0.4 * np.sin(2.0 * np.pi * x) + 0.5 * (x > 0.6))[None, None, :]
    d = O.make_desc(n1, 4, 4, 0.0, 0.0, 0.0, 1.0 / n1, 1.0, 1.0, metric=O.METRIC_MINKOWSKI, gam=gam,
                    cour=0.5, recon=O.RECON_PPM, riemann=O.FLUX_HLL, bc=(1, 1, 1, 1, 1, 1), floors=0)
    g = O.Grid(d)
    g.set(prim, bf)
    F = g.fluxes()
    p, _ = g.get()  # ghosts filled as the fluxes saw them
    j = k = NG + 1
    kap = (gam - 1.0) * p[1][k, j, :] / p[0][k, j, :] ** gam
    kl, kr = O.recon_line(O.RECON_PPM, kap)
    faces = np.arange(NG, NG + n1 + 1)  # x1-faces 0..n1: face i lies between cells i-1 and i
    ratio = F[0, 5][k, j, faces] / F[0, 0][k, j, faces]
    assert np.allclose(ratio, kr[faces - 1], rtol=1e-14, atol=0.0)
    # the downwind cell's left edge value is another number wherever kappa varies
    assert np.abs(kl[faces] / kr[faces - 1] - 1.0).max() > 1e-3
