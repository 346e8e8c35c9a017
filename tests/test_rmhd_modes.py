"""Pins of the test-side SRMHD eigenmodes (tests/rmhd_modes.py) against closed
forms: the entropy wave is at rest, the Alfven speed along x is
B^x / sqrt(w + B^2), field along x gives the sound and Alfven speeds as the
magnetosonic pair, field across x gives a fast speed with c^2 = vA^2 +
cs^2 (1 - vA^2) and a vanishing slow speed; eigenvectors solve the linear
system; the Jacobian of the flux of an unmagnetised state reduces to
relativistic hydrodynamics' sound speed."""
import math

import numpy as np

import rmhd_modes as M

GAM = 5.0 / 3.0


def _speeds(rho, p, B):
    w = rho + p / (GAM - 1.0) + p
    cs2 = GAM * p / w
    va2 = (B @ B) / (w + B @ B)
    return w, cs2, va2


def test_alfven_and_entropy_speeds_oblique_field():
    B = np.array([0.6, 0.4, 0.2])
    rho, p = 1.0, 0.5
    lam, R = M.modes(rho, p, B, GAM)
    w, cs2, va2 = _speeds(rho, p, B)
    assert abs(lam[3]) < 1e-12
    va_x = B[0] / math.sqrt(w + B @ B)
    assert abs(lam[5] - va_x) < 1e-12 and abs(lam[1] + va_x) < 1e-12
    UP, FP = M.jacobians(np.array([rho, p, 0, 0, 0, B[1], B[2]]), B[0], GAM)
    for m in range(7):
        r = R[:, m]
        assert np.abs(FP @ r - lam[m] * (UP @ r)).max() < 1e-12 * np.abs(UP @ r).max()


def test_field_along_and_across_x():
    rho, p = 1.0, 0.5
    B = np.array([0.8, 0.0, 0.0])
    lam, _ = M.modes(rho, p, B, GAM)
    w, cs2, va2 = _speeds(rho, p, B)
    pos = sorted(x for x in lam if x > 1e-9)
    want = sorted([math.sqrt(cs2), math.sqrt(va2)])
    # along x: the magnetosonic pair is {cs, vA} (the Alfven speed appears twice)
    assert abs(pos[-1] - max(want)) < 1e-12 and abs(pos[0] - min(want)) < 1e-12
    B = np.array([0.0, 0.8, 0.0])
    lam, _ = M.modes(rho, p, B, GAM)
    w, cs2, va2 = _speeds(rho, p, B)
    assert abs(lam[-1] - math.sqrt(va2 + cs2 * (1.0 - va2))) < 1e-12
    assert np.sum(np.abs(lam) < 1e-9) >= 3  # slow, Alfven and entropy at zero


def test_hydro_sound_speed():
    rho, p = 2.0, 0.3
    lam, _ = M.modes(rho, p, np.zeros(3), GAM)
    w = rho + p / (GAM - 1.0) + p
    assert abs(lam[-1] - math.sqrt(GAM * p / w)) < 1e-12
